"""Write the oracle's full Fock build G = J - K/2 of one (H2O)32 bead
(768 functions) to tests/golden/, as projections small enough to store.

The converged SCF of a 768-function bead is out of the oracle's reach (about
7e8 screened shell quartets per Fock build; tens of hours per build sequence
on the host cores), so the full-size check of the Fock build uses one build of
a density the oracle makes itself: the core-Hamiltonian guess of the bead
(one diagonalisation of h in the Loewdin basis, n_occ = 160), which is dense
and of SCF-like magnitude. Stored: G v_k for two seeded vectors, v_k^T G v_k,
tr(D G), the diagonal of G and two full rows. Only `oracle/` and the seeded
input generators are used. Usage:
    python tests/golden/make_fock_golden.py water32_spd_16beads 0
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

ROWS = (5, 501)
VEC_SEEDS = (3201, 3202)


def core_density(bas, Z, X):
    """The oracle's core-Hamiltonian guess density of one replica."""
    ob = O.OracleBasis.build(bas, Z, X)
    S, T, V = O.one_electron(ob, Z, X)
    Xo = O.orthogonaliser(S)
    return ob, O.core_guess(T + V, Xo, int(sum(int(z) for z in Z)) // 2)


def probe_vectors(n):
    return [np.random.default_rng(s).normal(size=n) for s in VEC_SEEDS]


def main():
    name = sys.argv[1]
    k = int(sys.argv[2])
    reps, kind = inputs.workload(name)
    bas = inputs.basis_set(kind)
    Z, X = reps.Z[k], reps.coords[k]
    ob, D = core_density(bas, Z, X)
    t = time.time()
    J, K, nq = O.jk(ob, D, 1e-12)
    secs = time.time() - t
    G = J - 0.5 * K
    vs = probe_vectors(ob.nbf)
    out = {
        "workload": name,
        "replica": k,
        "basis": kind,
        "source": "oracle/ (McMurchie-Davidson J and K over canonical quartets, Schwarz 1e-12), "
                  "written by tests/golden/make_fock_golden.py",
        "density": "oracle core-Hamiltonian guess of the replica (Loewdin basis, aufbau)",
        "nbf": int(ob.nbf),
        "coords_bohr": np.asarray(X).tolist(),
        "nquartets": int(nq),
        "tr_DG": float(np.sum(D * G)),
        "vec_seeds": list(VEC_SEEDS),
        "Gv": [(G @ v).tolist() for v in vs],
        "vGv": [float(v @ G @ v) for v in vs],
        "diag": np.diag(G).tolist(),
        "rows": {str(r): G[r].tolist() for r in ROWS},
        "oracle_seconds": secs,
        "oracle_threads": O.num_threads(),
    }
    path = os.path.join(HERE, f"{name}_rep{k}_fock.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(path, nq, secs, flush=True)


if __name__ == "__main__":
    main()
