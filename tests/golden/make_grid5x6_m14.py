"""Write grid5x6_m14_amps.json: oracle state-vector amplitudes of the 30-qubit,
14-cycle grid workload for its 16 seeded bitstring prefixes x 64 open
assignments. Calls only the oracle (FP64 state vector, Sec. 2-3)."""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synthetic.circuits import CONFIGS, config_circuit, random_bits  # noqa: E402


def prefixes(name):
    cfg = CONFIGS[name]
    c = config_circuit(name)
    oq = c.layout.open_qubits(cfg["n_open"])
    n_closed = c.n_qubits - len(oq)
    return c, oq, [list(random_bits(n_closed, cfg["bit_seed"] + i)) for i in range(cfg["prefixes"])]


def main():
    name = "grid5x6_m14"
    c, oq, pre = prefixes(name)
    psi = oracle.statevector(c)
    amps = [oracle.sv_amplitudes(c, oq, p, psi) for p in pre]
    out = {
        "cite": "Oracle FP64 state vector (Sec. 2 circuit rules, Sec. 3 Schroedinger method); "
                "workload grid5x6_m14 of synthetic.circuits.CONFIGS",
        "workload": name, "open_qubits": oq, "prefixes": [[int(b) for b in p] for p in pre],
        "norm": float(np.vdot(psi, psi).real),
        "amps_re": [[float(x.real) for x in a] for a in amps],
        "amps_im": [[float(x.imag) for x in a] for a in amps],
    }
    with open(os.path.join(HERE, f"{name}_amps.json"), "w") as fh:
        json.dump(out, fh)


if __name__ == "__main__":
    main()
