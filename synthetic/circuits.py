"""Seeded random-circuit generator in the shape of the paper's Sycamore family.

The rules follow Sec. 2 of the paper: ``m`` cycles, each a single-qubit layer
followed by a two-qubit layer, then one more single-qubit layer before
measurement. Single-qubit gates are drawn from {sqrt(X), sqrt(Y), sqrt(W)}:
uniformly in the first layer, and in every later layer uniformly from the two
gates that differ from the gate that qubit received in the previous layer.
Two-qubit layers follow the coupler pattern sequence A B C D C D A B, repeated.

Readings of what the paper leaves open (its layout figure is not available):

* Gate identifiers: 0 = sqrt(X), 1 = sqrt(Y), 2 = sqrt(W).
* Random numbers: SplitMix64 (Steele, Lea, Flood 2014), draws taken in the
  order (layer ascending, qubit ascending); a choice among c options is
  ``next() % c``.
* Rectangular grids: qubit (r, c) has id ``r * cols + c``. Pattern A pairs
  (r, c)-(r, c+1) with r + c even, B the same with r + c odd, C pairs
  (r, c)-(r+1, c) with r + c even, D the same with r + c odd.
* 53-site stand-in for the Sycamore chip: 9 rows of 6 sites on a diagonal
  lattice (even rows shifted half a site right), site (8, 5) removed. Site
  (i, j) of an even row couples to (i+1, j) and (i+1, j+1); of an odd row to
  (i+1, j-1) and (i+1, j). Classes: A = down-left couplers from even rows,
  B = down-left from odd rows, C = down-right from even rows, D = down-right
  from odd rows. Each class is a matching.
* A qubit untouched by the current pattern gets no two-qubit gate.
* fSim parameters theta = pi/2, phi = pi/6 on every coupler, no extra
  Z rotations.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple

import numpy as np

MASK64 = (1 << 64) - 1
PATTERN_SEQUENCE = "ABCDCDAB"


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood, OOPSLA 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def below(self, c: int) -> int:
        return self.next() % c


@dataclass
class Layout:
    """Qubit sites and the four coupler classes A-D (each a matching)."""

    name: str
    sites: List[Tuple[int, int]]
    classes: Dict[str, List[Tuple[int, int]]]
    corner: List[Tuple[int, int]]  # open-qubit candidates, in order

    @property
    def n_qubits(self) -> int:
        return len(self.sites)

    def qubit(self, site: Tuple[int, int]) -> int:
        return self.sites.index(tuple(site))

    def open_qubits(self, n_open: int) -> List[int]:
        if n_open > len(self.corner):
            raise ValueError("too many open qubits for this layout")
        return [self.qubit(s) for s in self.corner[:n_open]]


def grid_layout(rows: int, cols: int) -> Layout:
    sites = [(r, c) for r in range(rows) for c in range(cols)]
    qid = {s: i for i, s in enumerate(sites)}
    classes = {k: [] for k in "ABCD"}
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                classes["A" if (r + c) % 2 == 0 else "B"].append((qid[(r, c)], qid[(r, c + 1)]))
            if r + 1 < rows:
                classes["C" if (r + c) % 2 == 0 else "D"].append((qid[(r, c)], qid[(r + 1, c)]))
    corner = [(0, cols - 3), (0, cols - 2), (0, cols - 1), (1, cols - 2), (1, cols - 1),
              (2, cols - 1), (1, cols - 3), (2, cols - 2)]
    corner = [s for s in corner if s in qid]
    return Layout(f"grid{rows}x{cols}", sites, classes, corner)


def diagonal53_layout() -> Layout:
    rows, cols = 9, 6
    removed = (8, 5)
    sites = [(i, j) for i in range(rows) for j in range(cols) if (i, j) != removed]
    qid = {s: k for k, s in enumerate(sites)}
    classes = {k: [] for k in "ABCD"}
    for (i, j) in sites:
        if i + 1 >= rows:
            continue
        if i % 2 == 0:
            left, right = (i + 1, j), (i + 1, j + 1)
        else:
            left, right = (i + 1, j - 1), (i + 1, j)
        if left in qid:
            classes["A" if i % 2 == 0 else "B"].append((qid[(i, j)], qid[left]))
        if right in qid:
            classes["C" if i % 2 == 0 else "D"].append((qid[(i, j)], qid[right]))
    corner = [(0, 3), (0, 4), (0, 5), (1, 4), (1, 5), (2, 5), (1, 3), (2, 4)]
    return Layout("diag53", sites, classes, corner)


@dataclass
class Circuit:
    """A random circuit as gate identifiers; no matrices.

    ``gates_1q[t][q]`` is the identifier of the single-qubit gate on qubit q in
    single-qubit layer t (t = 0..m, layer m is the one before measurement).
    ``pairs[t]`` lists the (qa, qb) couplers of two-qubit layer t (t < m),
    with qa < qb.
    """

    n_qubits: int
    n_cycles: int
    gates_1q: List[List[int]]
    pairs: List[List[Tuple[int, int]]]
    theta: float = math.pi / 2
    phi: float = math.pi / 6
    layout: Layout | None = field(default=None, repr=False)

    def flat(self):
        """Flat arrays in the order the C interface expects."""
        g = np.asarray(self.gates_1q, dtype=np.int8).reshape(self.n_cycles + 1, self.n_qubits)
        offs = [0]
        flat_pairs: List[int] = []
        for layer in self.pairs:
            for a, b in layer:
                flat_pairs += [a, b]
            offs.append(len(flat_pairs) // 2)
        return (np.ascontiguousarray(g), np.asarray(offs, dtype=np.int32),
                np.asarray(flat_pairs if flat_pairs else [0], dtype=np.int32))

    def n_gates_2q(self) -> int:
        return sum(len(p) for p in self.pairs)


def random_circuit(layout: Layout, n_cycles: int, seed: int,
                   theta: float = math.pi / 2, phi: float = math.pi / 6) -> Circuit:
    rng = SplitMix64(seed)
    n = layout.n_qubits
    gates: List[List[int]] = []
    prev = [-1] * n
    for t in range(n_cycles + 1):
        layer = []
        for q in range(n):
            if prev[q] < 0:
                g = rng.below(3)
            else:
                others = [x for x in range(3) if x != prev[q]]
                g = others[rng.below(2)]
            layer.append(g)
            prev[q] = g
        gates.append(layer)
    pairs = []
    for t in range(n_cycles):
        cls = PATTERN_SEQUENCE[t % len(PATTERN_SEQUENCE)]
        pairs.append([(min(a, b), max(a, b)) for a, b in layout.classes[cls]])
    return Circuit(n, n_cycles, gates, pairs, theta, phi, layout)


def random_bits(n_bits: int, seed: int) -> np.ndarray:
    rng = SplitMix64(seed)
    return np.asarray([rng.below(2) for _ in range(n_bits)], dtype=np.uint8)


def random_uniform(shape: Sequence[int], seed: int) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of SplitMix64 draws, in
    row-major order (random numbers a method consumes are inputs)."""
    rng = SplitMix64(seed)
    n = int(np.prod(shape))
    return (np.asarray([rng.next() >> 11 for _ in range(n)], dtype=np.float64) *
            (1.0 / 9007199254740992.0)).reshape(shape)


def random_complex(shape: Sequence[int], seed: int = 7, dtype=np.complex128) -> np.ndarray:
    """N(0,1) complex test tensor (real and imaginary parts independent)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(dtype)


# Workload configurations (circuit shapes, seeds, batch shapes). Names say what
# each workload is; sizes are the paper-shaped ones.
CONFIGS = {
    "grid4x4_m8": dict(layout=("grid", 4, 4), cycles=8, seed=1, n_open=0,
                       bitstrings=64, bit_seed=101, cw_limit=None),
    "grid5x6_m14": dict(layout=("grid", 5, 6), cycles=14, seed=2, n_open=6,
                        prefixes=16, bit_seed=201, n_sliced=8, cw_limit=None),
    "diag53_m12": dict(layout=("diag53",), cycles=12, seed=3, n_open=6,
                       bit_seed=301, cw_limit=28, n_sliced=10),
    "diag53_m14": dict(layout=("diag53",), cycles=14, seed=4, n_open=6,
                       bit_seed=401, cw_limit=30),
    "diag53_m20": dict(layout=("diag53",), cycles=20, seed=5, n_open=6,
                       bit_seed=501, cw_limit=30),
}


def make_layout(spec) -> Layout:
    if spec[0] == "grid":
        return grid_layout(spec[1], spec[2])
    if spec[0] == "diag53":
        return diagonal53_layout()
    raise ValueError(spec)


def config_circuit(name: str) -> Circuit:
    cfg = CONFIGS[name]
    return random_circuit(make_layout(cfg["layout"]), cfg["cycles"], cfg["seed"])
