"""Write <workload>_slices.json: oracle (FP64 pairwise contraction, Supp. A.1)
values of a few slices of a workload, each with the 2^n_open open amplitudes.

The sub-network of a slice is fixed by its sliced wire segments; the oracle
contracts it along the given order (a schedule only: the value does not depend
on it, Sec. 3). Order and sliced wire segments are read from
<workload>_scheme.json; the values are the oracle's alone (this script calls
nothing but the oracle and the seeded input generators).

    python make_stored_slices.py diag53_m14 0 1

The 53-qubit, 14-cycle slices reach 2^30-entry FP64 tensors (16 GiB each, two
alive at a time), so the run needs about 40 GB of host memory.
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from synthetic.circuits import CONFIGS, config_circuit, random_bits  # noqa: E402


def main(name: str, slices):
    sch = json.load(open(os.path.join(HERE, f"{name}_scheme.json")))
    cfg = CONFIGS[name]
    c = config_circuit(name)
    oq = c.layout.open_qubits(cfg["n_open"])
    cb = list(random_bits(c.n_qubits - len(oq), cfg["bit_seed"]))
    net = oracle.build_network(c, oq, cb)
    wires = [tuple(w) for w in sch["sliced_wires"]]
    order = [tuple(p) for p in sch["order"]]
    out = {"cite": "Oracle FP64 pairwise contraction (Supp. A.1) of the listed slices; "
                   "slice s fixes sliced wire j to bit j of s (Supp. A.1 'Slicing')",
           "workload": name, "sliced_wires": sch["sliced_wires"], "threads": oracle_threads(),
           "slices": {}}
    path = os.path.join(HERE, f"{name}_slices.json")
    for sid in slices:
        t = time.time()
        v = oracle.contract(net, order, oracle.slice_assignment(wires, sid)).reshape(-1)
        out["slices"][str(sid)] = {"re": [float(x.real) for x in v], "im": [float(x.imag) for x in v],
                                   "seconds": time.time() - t}
        print(name, sid, f"{time.time() - t:.1f} s", flush=True)
        with open(path, "w") as fh:
            json.dump(out, fh)


def oracle_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


if __name__ == "__main__":
    main(sys.argv[1], [int(x) for x in sys.argv[2:]] or [0, 1])
