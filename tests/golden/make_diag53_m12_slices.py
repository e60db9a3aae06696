"""Write diag53_m12_slices.json: oracle (FP64 pairwise contraction, Supp. A.1)
values of a few slices of the 53-qubit, 12-cycle workload, with the 64 open
amplitudes of each.

The sub-network of a slice is fixed by its sliced wire segments; the oracle
contracts it along the given order (a schedule only: the value does not
depend on it, Sec. 3). Order and sliced wire segments are read from
diag53_m12_scheme.json (written with the same workload by the library's
planner); the values are the oracle's alone. Run: python make_diag53_m12_slices.py
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synthetic.circuits import CONFIGS, config_circuit, random_bits  # noqa: E402

NAME = "diag53_m12"
SLICES = [0, 1]


def main():
    sch = json.load(open(os.path.join(HERE, f"{NAME}_scheme.json")))
    cfg = CONFIGS[NAME]
    c = config_circuit(NAME)
    oq = c.layout.open_qubits(cfg["n_open"])
    cb = list(random_bits(c.n_qubits - len(oq), cfg["bit_seed"]))
    net = oracle.build_network(c, oq, cb)
    wires = [tuple(w) for w in sch["sliced_wires"]]
    order = [tuple(p) for p in sch["order"]]
    out = {"cite": "Oracle FP64 pairwise contraction (Supp. A.1) of the listed slices; "
                   "slice s fixes sliced wire j to bit j of s (Supp. A.1 'Slicing')",
           "workload": NAME, "sliced_wires": sch["sliced_wires"], "slices": {}}
    for sid in SLICES:
        t = time.time()
        v = oracle.contract(net, order, oracle.slice_assignment(wires, sid)).reshape(-1)
        out["slices"][str(sid)] = {"re": [float(x.real) for x in v], "im": [float(x.imag) for x in v],
                                   "seconds": time.time() - t}
        print(sid, time.time() - t, flush=True)
    with open(os.path.join(HERE, f"{NAME}_slices.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
