"""Write <workload>_scheme.json: the contraction order and sliced wire segments
of the library's plan for a workload (the planner options of bench.py).

This is schedule input for the oracle, not a value: the value of a
(sub-)network does not depend on the order (Sec. 3), and the sliced wire
segments only name which wires a slice fixes (Supp. A.1, "Slicing"). Every
expected value is computed from it by make_stored_slices.py, which calls only
the oracle. Run: python make_scheme.py diag53_m14
"""

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import paper_2005_06787_gb300 as P  # noqa: E402
from bench import plan_options, workload_inputs  # noqa: E402


def main(name: str, extra: dict):
    c, oq, cb = workload_inputs(name)
    net = P.tn_build_network(c, oq, cb)
    t = time.time()
    plan = P.tn_plan_create(net, **dict(plan_options(name), **extra))
    order, sl = P.tn_plan_export(plan)
    info = P.tn_plan_info(plan)
    _, _, q, s = net.info()
    out = {"workload": name,
           "note": "contraction order and sliced wire segments of the library's plan for this "
                   "workload (plan_options in bench.py); schedule input for the oracle",
           "planner_options_beyond_plan_options": extra,
           "log2_tc": info["log2_tc"], "cw": info["cw"], "n_sliced": info["n_sliced"],
           "order": [[int(a), int(b)] for a, b in order],
           "sliced_wires": [[int(q[e]), int(s[e])] for e in sl]}
    with open(os.path.join(HERE, f"{name}_scheme.json"), "w") as fh:
        json.dump(out, fh)
    print(name, f"log2 tc {info['log2_tc']:.3f}, cw {info['cw']}, {info['n_sliced']} sliced, "
                f"{time.time() - t:.1f} s")


if __name__ == "__main__":
    # optional second argument: planner options beyond bench.plan_options, as
    # JSON, e.g. the stored 20-cycle plan of total cost 2^61.99 (all 386 start
    # clusters, about an hour on 8 host cores):
    #   python make_scheme.py diag53_m20 '{"stem_starts": 386, "anneal_iters": 1200000,
    #       "restarts": 1, "slice_restarts": 0, "max_sliced": 64}'
    main(sys.argv[1] if len(sys.argv) > 1 else "diag53_m14",
         json.loads(sys.argv[2]) if len(sys.argv) > 2 else {})
