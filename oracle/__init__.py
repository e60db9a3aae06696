"""Oracle for the stem contraction: plain FP64 CPU code, test infrastructure.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline leg
may import this package. It shares no code with the GPU library
(``paper_2005_06787_gb300``) and imports nothing from it; the two meet only in
the seeded inputs of ``synthetic``.

Contents and the passages they follow:

* ``gate_1q``, ``fsim``: the gate matrices of Sec. 2 (computed in ``oracle.c``).
* ``statevector``, ``sv_amplitudes``: Schroedinger evolution (Sec. 3) of the
  Sec. 2 circuit, optionally with |v><v| on chosen wire segments: fixing a
  sliced edge (Supp. A.1, "Slicing") to v.
* ``build_network``: the circuit as a tensor network (Sec. 3, Supp. A.1):
  one tensor per |0>, gate and closed-qubit projector, one edge per wire
  segment, open edges on the open qubits' last segments.
* ``build_hypernetwork``: the same circuit as a multi-hypergraph (Supp. A.1
  defines networks as hypergraphs; Sec. 3 names hyperedges for diagonal gate
  parts, after BIS+18). With theta = pi/2, fSim(pi/2, phi) is the wire swap
  times diag(1, -i, -i, e^{-i phi}): each two-qubit gate becomes a rank-2
  diagonal tensor on the two current wire indices, which the wires then
  exchange; an index is created only by |0> and single-qubit gates.
* ``contract``: sequential pairwise contraction (Sec. 3, Schroedinger method;
  Supp. A.1 contraction trees) with ``orc_contract`` as each step: a step
  keeps E*_AB, the edges of the pair that are open or held by another
  remaining tensor (in a graph: the edges of exactly one of the two); sliced
  edges are fixed by indexing, and ``contract_sliced_sum`` sums subtasks
  (Supp. A.1, "Slicing").
* ``feynman``: T_H[b] as the literal sum of path values (Supp. A.1).
* ``tree_cost``: tc and cw of a contraction scheme (Supp. A.1: per step
  2^|E_AB| and |E*_AB|; tc sums, cw maxes; slicing multiplies tc by 2^|E_s|).
* ``linear_xeb``: 2^n <p> - 1 (Sec. 2).
* ``frugal_sample``: frugal rejection sampling over amplitude batches (Sec.
  2, after the method the paper cites as MFI+18): candidate x is accepted
  with probability min(1, 2^n p(x) / M); a batch yields its first accepted
  candidate in a random visiting order.

Leaf numbering (shared convention, each side implements it itself): leaves
0..n-1 are |0> on qubits 0..n-1; then for each cycle t < m the single-qubit
gates of layer t on qubits 0..n-1 followed by the two-qubit gates of layer t
in listed order; then the final single-qubit layer on qubits 0..n-1; then
one projector <b_q| per closed qubit in ascending q. An edge is the wire
segment (q, s): segment s of qubit q follows the s-th gate acting on q.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_c128p = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-shared", "-fPIC",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_gate_1q.argtypes = [ctypes.c_int, _c128p]
        L.orc_gate_1q.restype = ctypes.c_int
        L.orc_fsim.argtypes = [ctypes.c_double, ctypes.c_double, _c128p]
        L.orc_fsim.restype = None
        L.orc_statevector.argtypes = [ctypes.c_int, ctypes.c_int, _i8p, _i32p, _i32p,
                                      ctypes.c_double, ctypes.c_double, _i32p, _i32p, _i8p,
                                      ctypes.c_int, _c128p]
        L.orc_statevector.restype = ctypes.c_int
        L.orc_contract.argtypes = [_c128p, ctypes.c_int, _i64p, _c128p, ctypes.c_int, _i64p,
                                   _c128p, ctypes.c_int, _i64p]
        L.orc_contract.restype = ctypes.c_int
        L.orc_feynman.argtypes = [ctypes.c_int, _i32p, _i32p, _i32p, _i64p, _c128p,
                                  ctypes.c_int, _i32p, ctypes.c_int, _c128p]
        L.orc_feynman.restype = ctypes.c_int
        _lib = L
    return _lib


# ----------------------------------------------------------------------------
# gates (Sec. 2)

def gate_1q(gid: int) -> np.ndarray:
    g = np.zeros(4, dtype=np.complex128)
    if lib().orc_gate_1q(int(gid), g) != 0:
        raise ValueError(f"unknown gate id {gid}")
    return g.reshape(2, 2)


def fsim(theta: float, phi: float) -> np.ndarray:
    f = np.zeros(16, dtype=np.complex128)
    lib().orc_fsim(float(theta), float(phi), f)
    return f.reshape(4, 4)


# ----------------------------------------------------------------------------
# state vector (Sec. 2, Sec. 3)

def _projector_arrays(projectors: Optional[Dict[Tuple[int, int], int]]):
    items = sorted((projectors or {}).items())
    pq = np.asarray([k[0] for k, _ in items] or [0], dtype=np.int32)
    ps = np.asarray([k[1] for k, _ in items] or [0], dtype=np.int32)
    pv = np.asarray([v for _, v in items] or [0], dtype=np.int8)
    return pq, ps, pv, len(items)


def statevector(circuit, projectors: Optional[Dict[Tuple[int, int], int]] = None) -> np.ndarray:
    """Final state C|0..0> (qubit 0 = most significant bit of the index)."""
    g, offs, pairs = circuit.flat()
    n = circuit.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    pq, ps, pv, npj = _projector_arrays(projectors)
    rc = lib().orc_statevector(n, circuit.n_cycles, g.reshape(-1), offs, pairs,
                               circuit.theta, circuit.phi, pq, ps, pv, npj, psi)
    if rc != 0:
        raise ValueError("orc_statevector rejected the circuit")
    return psi


def basis_index(n: int, bits_by_qubit: Sequence[int]) -> int:
    x = 0
    for q in range(n):
        x = 2 * x + int(bits_by_qubit[q])
    return x


def sv_amplitudes(circuit, open_qubits: Sequence[int], closed_bits: Sequence[int],
                  psi: Optional[np.ndarray] = None,
                  projectors: Optional[Dict[Tuple[int, int], int]] = None) -> np.ndarray:
    """Amplitudes <x|C|0> for every assignment of the open qubits (first open
    qubit = most significant bit of the result index); the closed qubits, in
    ascending order, take ``closed_bits``."""
    n = circuit.n_qubits
    if psi is None:
        psi = statevector(circuit, projectors)
    closed = [q for q in range(n) if q not in set(open_qubits)]
    if len(closed) != len(closed_bits):
        raise ValueError("closed_bits must give one bit per closed qubit")
    k = len(open_qubits)
    out = np.zeros(1 << k, dtype=np.complex128)
    for b in range(1 << k):
        bits = [0] * n
        for q, v in zip(closed, closed_bits):
            bits[q] = int(v)
        for i, q in enumerate(open_qubits):
            bits[q] = (b >> (k - 1 - i)) & 1
        out[b] = psi[basis_index(n, bits)]
    return out


# ----------------------------------------------------------------------------
# tensor network (Sec. 3, Supp. A.1)

Edge = Tuple[int, int]  # wire segment (qubit, segment)


@dataclass
class Network:
    tensors: List[np.ndarray]            # complex128, shape (2,)*rank
    edges: List[List[Edge]]              # per tensor, ordered
    open_edges: List[Edge]               # in open-qubit order
    kinds: List[str] = field(default_factory=list)

    def all_edges(self) -> List[Edge]:
        seen = []
        s = set()
        for el in self.edges:
            for e in el:
                if e not in s:
                    s.add(e)
                    seen.append(e)
        return seen


def build_network(circuit, open_qubits: Sequence[int], closed_bits: Sequence[int]) -> Network:
    n, m = circuit.n_qubits, circuit.n_cycles
    open_set = set(open_qubits)
    closed = [q for q in range(n) if q not in open_set]
    if len(closed) != len(closed_bits):
        raise ValueError("closed_bits must give one bit per closed qubit")
    seg = [0] * n
    tensors: List[np.ndarray] = []
    edges: List[List[Edge]] = []
    kinds: List[str] = []

    def add(t, el, kind):
        tensors.append(np.ascontiguousarray(t, dtype=np.complex128))
        edges.append(el)
        kinds.append(kind)

    for q in range(n):
        add(np.array([1.0, 0.0]), [(q, 0)], "zero")
    F = fsim(circuit.theta, circuit.phi)
    for t in range(m + 1):
        for q in range(n):
            G = gate_1q(circuit.gates_1q[t][q])
            # T[in, out] = G[out, in]
            add(G.T.copy(), [(q, seg[q]), (q, seg[q] + 1)], "1q")
            seg[q] += 1
        if t == m:
            break
        for (qa, qb) in circuit.pairs[t]:
            # T[ia, ib, oa, ob] = F[(oa, ob), (ia, ib)]
            T = F.reshape(2, 2, 2, 2).transpose(2, 3, 0, 1)
            add(T, [(qa, seg[qa]), (qb, seg[qb]), (qa, seg[qa] + 1), (qb, seg[qb] + 1)], "2q")
            seg[qa] += 1
            seg[qb] += 1
    for q, v in zip(closed, closed_bits):
        add(np.array([1.0, 0.0]) if int(v) == 0 else np.array([0.0, 1.0]), [(q, seg[q])], "proj")
    open_edges = [(q, seg[q]) for q in open_qubits]
    return Network(tensors, edges, open_edges, kinds)


def build_hypernetwork(circuit, open_qubits: Sequence[int], closed_bits: Sequence[int]) -> Network:
    """The circuit's hypergraph network (Supp. A.1, Sec. 3): indices are
    created by |0> and single-qubit gates only; each fSim(pi/2, phi) is the
    rank-2 tensor d[x_a, x_b] = fSim[(x_b, x_a), (x_a, x_b)] on the two
    current wire indices, after which qubits a and b carry each other's
    index. Index (q, j) is the one qubit q's j-th gate created ((q, 0): its
    |0>). Raises ValueError unless theta = pi/2."""
    n, m = circuit.n_qubits, circuit.n_cycles
    if abs(np.cos(circuit.theta)) > 1e-12:
        raise ValueError("hyperedge network needs fSim(pi/2, phi): a wire swap times a diagonal gate")
    open_set = set(open_qubits)
    closed = [q for q in range(n) if q not in open_set]
    if len(closed) != len(closed_bits):
        raise ValueError("closed_bits must give one bit per closed qubit")
    cur: List[Edge] = [(q, 0) for q in range(n)]
    made = [0] * n
    tensors: List[np.ndarray] = []
    edges: List[List[Edge]] = []
    kinds: List[str] = []

    def add(t, el, kind):
        tensors.append(np.ascontiguousarray(t, dtype=np.complex128))
        edges.append(el)
        kinds.append(kind)

    for q in range(n):
        add(np.array([1.0, 0.0]), [cur[q]], "zero")
    F = fsim(circuit.theta, circuit.phi).reshape(2, 2, 2, 2)  # [ya, yb, xa, xb]
    D = np.array([[F[xb, xa, xa, xb] for xb in range(2)] for xa in range(2)])
    for t in range(m + 1):
        for q in range(n):
            G = gate_1q(circuit.gates_1q[t][q])
            made[q] += 1
            out = (q, made[q])
            add(G.T.copy(), [cur[q], out], "1q")  # T[in, out] = G[out, in]
            cur[q] = out
        if t == m:
            break
        for (qa, qb) in circuit.pairs[t]:
            add(D, [cur[qa], cur[qb]], "diag")
            cur[qa], cur[qb] = cur[qb], cur[qa]
    for q, v in zip(closed, closed_bits):
        add(np.array([1.0, 0.0]) if int(v) == 0 else np.array([0.0, 1.0]), [cur[q]], "proj")
    return Network(tensors, edges, [cur[q] for q in open_qubits], kinds)


def fix_edges(net: Network, sliced: Dict[Edge, int]) -> Network:
    """Sub-network with each sliced edge fixed to its value (Supp. A.1)."""
    tensors, edges = [], []
    for T, el in zip(net.tensors, net.edges):
        idx = []
        keep = []
        for e in el:
            if e in sliced:
                idx.append(int(sliced[e]))
            else:
                idx.append(slice(None))
                keep.append(e)
        tensors.append(np.ascontiguousarray(T[tuple(idx)]))
        edges.append(keep)
    for e in sliced:
        if e in net.open_edges:
            raise ValueError("an open edge cannot be sliced")
    return Network(tensors, edges, list(net.open_edges), list(net.kinds))


def _i64_labels(el: Sequence[Edge]) -> np.ndarray:
    return np.asarray([q * 1_000_003 + s for q, s in el] or [0], dtype=np.int64)


def contract_pair(A: np.ndarray, ea: List[Edge], B: np.ndarray, eb: List[Edge],
                  keep: Optional[Sequence[Edge]] = None) -> Tuple[np.ndarray, List[Edge]]:
    """Contract A and B. Without ``keep`` (a graph): the shared edges are
    summed and the output edges are A's unshared edges then B's. With
    ``keep`` (E*_AB of Supp. A.1): the output edges are the edges of A, then
    those of B not in A, that are in ``keep``; every other edge is summed."""
    sb = set(eb)
    sa = set(ea)
    if keep is None:
        ec = [e for e in ea if e not in sb] + [e for e in eb if e not in sa]
    else:
        kp = set(keep)
        ec = [e for e in ea if e in kp] + [e for e in eb if e in kp and e not in sa]
    C = np.zeros(1 << len(ec), dtype=np.complex128)
    A1 = np.ascontiguousarray(A.reshape(-1))
    B1 = np.ascontiguousarray(B.reshape(-1))
    rc = lib().orc_contract(A1, len(ea), _i64_labels(ea), B1, len(eb), _i64_labels(eb),
                            C, len(ec), _i64_labels(ec))
    if rc != 0:
        raise ValueError("orc_contract rejected the edge lists")
    return C.reshape((2,) * len(ec)) if ec else C.reshape(()), ec


def contract(net: Network, order: Optional[Sequence[Tuple[int, int]]] = None,
             sliced: Optional[Dict[Edge, int]] = None) -> np.ndarray:
    """Value of the (sub-)network as a tensor over the open edges, axes in
    open-edge order. ``order`` is an SSA list of pairs: leaves are 0..N-1 and
    the k-th contraction creates tensor N+k. Without an order the tensors are
    folded left in leaf order. The value does not depend on the order
    (Sec. 3); the order only sets the cost."""
    if sliced:
        net = fix_edges(net, sliced)
    live: Dict[int, Tuple[np.ndarray, List[Edge]]] = {
        i: (T, list(el)) for i, (T, el) in enumerate(zip(net.tensors, net.edges))}
    N = len(net.tensors)
    if order is None:
        order = []
        cur = 0
        for i in range(1, N):
            order.append((cur, i))
            cur = N + i - 1
    nid = N
    opn = set(net.open_edges)
    holders: Dict[Edge, int] = {}  # number of remaining tensors holding each edge
    for _, el in live.values():
        for e in el:
            holders[e] = holders.get(e, 0) + 1
    for (a, b) in order:
        if a not in live or b not in live or a == b:
            raise ValueError(f"invalid contraction pair ({a}, {b})")
        A, ea = live.pop(a)
        B, eb = live.pop(b)
        for e in ea + eb:
            holders[e] -= 1
        # E*_AB: the pair's edges that are open or held by a remaining tensor
        keep = [e for e in set(ea) | set(eb) if e in opn or holders[e] > 0]
        C, ec = contract_pair(A, ea, B, eb, keep=keep)
        for e in ec:
            holders[e] += 1
        live[nid] = (C, ec)
        nid += 1
    if len(live) != 1:
        raise ValueError("the order does not contract the network to one tensor")
    (T, el), = live.values()
    if sorted(el) != sorted(net.open_edges):
        raise ValueError("the final tensor does not carry exactly the open edges")
    perm = [el.index(e) for e in net.open_edges]
    return np.transpose(T, perm) if perm else T


def slice_assignment(sliced_edges: Sequence[Edge], s: int) -> Dict[Edge, int]:
    """Slice id s fixes sliced edge j to bit j of s (least significant = j 0)."""
    return {e: (s >> j) & 1 for j, e in enumerate(sliced_edges)}


def contract_sliced_sum(net: Network, sliced_edges: Sequence[Edge],
                        order=None, slices: Optional[Sequence[int]] = None) -> np.ndarray:
    """Sum of the sub-network values over the listed slices (default: all),
    Supp. A.1 'Slicing'."""
    ids = range(1 << len(sliced_edges)) if slices is None else slices
    acc = None
    for s in ids:
        v = contract(net, order, slice_assignment(sliced_edges, s))
        acc = v if acc is None else acc + v
    return acc


def feynman(net: Network, sliced: Optional[Dict[Edge, int]] = None) -> np.ndarray:
    if sliced:
        net = fix_edges(net, sliced)
    labels = net.all_edges()
    for e in net.open_edges:
        if e not in labels:
            labels.append(e)
    eid = {e: i for i, e in enumerate(labels)}
    ranks = np.asarray([len(el) for el in net.edges], dtype=np.int32)
    offs = np.zeros(len(ranks), dtype=np.int32)
    offs[1:] = np.cumsum(ranks)[:-1]
    flat = np.asarray([eid[e] for el in net.edges for e in el] or [0], dtype=np.int32)
    sizes = [T.size for T in net.tensors]
    voff = np.zeros(len(sizes), dtype=np.int64)
    voff[1:] = np.cumsum(sizes)[:-1]
    vals = np.ascontiguousarray(np.concatenate([T.reshape(-1) for T in net.tensors]))
    opn = np.asarray([eid[e] for e in net.open_edges] or [0], dtype=np.int32)
    out = np.zeros(1 << len(net.open_edges), dtype=np.complex128)
    rc = lib().orc_feynman(len(ranks), ranks, offs, flat, voff, vals, len(labels), opn,
                           len(net.open_edges), out)
    if rc != 0:
        raise ValueError("orc_feynman rejected the network (too many edges?)")
    return out.reshape((2,) * len(net.open_edges)) if net.open_edges else out.reshape(())


# ----------------------------------------------------------------------------
# cost of a contraction scheme (Supp. A.1)

def tree_cost(edges: List[List[Edge]], open_edges: Sequence[Edge],
              order: Sequence[Tuple[int, int]], sliced: Sequence[Edge] = ()) -> Tuple[int, int]:
    """tc((E_s, T)) = 2^|E_s| * sum_u 2^|E_u| and cw = max_u |E*_u| over the
    internal nodes u of the tree given as an SSA pair list."""
    sl = set(sliced)
    live = {i: set(e for e in el if e not in sl) for i, el in enumerate(edges)}
    opn = set(open_edges)
    nid = len(edges)
    tc = 0
    cw = 0
    for (a, b) in order:
        ea, eb = live.pop(a), live.pop(b)
        e_ab = ea | eb
        elsewhere = set()
        for el in live.values():
            elsewhere |= el
        e_star = {e for e in e_ab if e in opn or e in elsewhere}
        tc += 1 << len(e_ab)
        cw = max(cw, len(e_star))
        live[nid] = e_star
        nid += 1
    return tc << len(sl), cw


def linear_xeb(probs: np.ndarray, n_qubits: int) -> float:
    """Sec. 2: 2^n <p_I(x)> - 1 over the sampled bitstrings' ideal p."""
    return float((2.0 ** n_qubits) * np.mean(probs) - 1.0)


def frugal_sample(amps: np.ndarray, n_qubits: int, M: float, u: np.ndarray,
                  key: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Frugal rejection sampling (Sec. 2): for batch b and candidate j,
    p = |amps[b, j]|^2 and the candidate is accepted when
    u[b, j] < 2^n p / M (the acceptance probability min(1, 2^n p / M) for u
    uniform in [0, 1)). The batch's sample is the accepted candidate with the
    smallest key[b, j] (keys uniform: a random visiting order, first accepted
    wins; equal keys go to the lower j), or -1 when none is accepted.

    The acceptance test is evaluated in FP64 as ((re*re + im*im) * 2^n) / M
    with each operation rounded separately. Returns (index [B], accepted
    count [B]), both int64."""
    a = np.asarray(amps, dtype=np.complex128)
    B, K = a.shape
    re, im = a.real.copy(), a.imag.copy()
    p = re * re + im * im
    thr = (p * (2.0 ** n_qubits)) / float(M)
    acc = np.asarray(u, dtype=np.float64) < thr
    idx = np.full(B, -1, dtype=np.int64)
    cnt = acc.sum(axis=1).astype(np.int64)
    keys = np.asarray(key, dtype=np.float64)
    for b in range(B):
        best = None
        for j in range(K):
            if acc[b, j] and (best is None or keys[b, j] < keys[b, best]):
                best = j
        if best is not None:
            idx[b] = best
    return idx, cnt
