"""Write oracle energies and gradients of selected replicas of the full-size
workloads to tests/golden/*.json (the oracle takes minutes to hours per
replica at these sizes, so the parity tests read stored values).

Only `oracle/` and the seeded input generators are used. Usage:
    python tests/golden/make_golden.py water8_spd_32beads 0 17
    python tests/golden/make_golden.py da_images_24 0 13
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1601_02713_gb300 import inputs  # noqa: E402


def main():
    name = sys.argv[1]
    idx = [int(x) for x in sys.argv[2:]]
    reps, kind = inputs.workload(name)
    bas = inputs.basis_set(kind)
    for k in idx:
        Z, X = reps.Z[k], reps.coords[k]
        t = time.time()
        E, G, res = O.rhf_energy_gradient(bas, Z, X)
        out = {
            "workload": name,
            "replica": k,
            "basis": kind,
            "source": "oracle/ (McMurchie-Davidson RHF, Schwarz 1e-12, |dE|<1e-10, max|e|<1e-8), "
                      "written by tests/golden/make_golden.py",
            "natom": int(len(Z)),
            "Z": [int(z) for z in Z],
            "coords_bohr": np.asarray(X).tolist(),
            "energy": float(E),
            "gradient": np.asarray(G).tolist(),
            "iterations": int(res.iterations),
            "converged": bool(res.converged),
            "homo_lumo_gap": float(res.homo_lumo_gap),
            "oracle_seconds": time.time() - t,
            "oracle_threads": O.num_threads(),
        }
        path = os.path.join(HERE, f"{name}_rep{k}.json")
        with open(path, "w") as fh:
            json.dump(out, fh, indent=1)
        print(path, E, out["oracle_seconds"], flush=True)


if __name__ == "__main__":
    main()
