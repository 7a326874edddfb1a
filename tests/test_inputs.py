"""The seeded input generators: shapes, determinism and the geometric rules
the workloads are defined by (bond lengths and angles of the water monomer,
minimum O-O distances of the packings, bead and MD-step displacement sizes,
atom counts of the ragged Diels-Alder images)."""
import numpy as np

from paper_1601_02713_gb300 import inputs

A = inputs.ANGSTROM_TO_BOHR


def _waters(Z, X):
    O = X[Z == 8]
    H = X[Z == 1].reshape(-1, 2, 3)
    return O, H


def test_monomer_geometry():
    Z, X = inputs.small_molecule("water")
    d1, d2 = np.linalg.norm(X[1] - X[0]) / A, np.linalg.norm(X[2] - X[0]) / A
    ang = np.degrees(np.arccos((X[1] - X[0]) @ (X[2] - X[0]) / (d1 * d2 * A * A)))
    assert abs(d1 - 0.957) < 1e-9 and abs(d2 - 0.957) < 1e-9 and abs(ang - 104.5) < 1e-6


def test_workloads_are_deterministic_and_sized():
    for name, nrep, natom, nbf in [("water2_min_4beads", 4, 6, 14), ("water8_spd_32beads", 32, 24, 192),
                                   ("water32_spd_16beads", 16, 96, 768)]:
        r1, kind = inputs.workload(name)
        r2, _ = inputs.workload(name)
        Z, X = r1.stacked()
        assert X.shape == (nrep, natom, 3)
        np.testing.assert_array_equal(X, r2.stacked()[1])
        assert inputs.nbf_of(inputs.basis_set(kind), Z) == nbf


def test_cluster_packing_rules():
    Z, X = inputs.water_cluster_geometry(8, 2)
    O, H = _waters(Z, X)
    d = np.linalg.norm(O[:, None] - O[None], axis=-1)
    np.fill_diagonal(d, np.inf)
    assert d.min() >= 2.6 - 1e-9
    # every O after the first is 2.9 A from some earlier O
    for k in range(1, len(O)):
        assert np.min(np.abs(np.linalg.norm(O[:k] - O[k], axis=1) - 2.9)) < 1e-9
    for o, hh in zip(O, H):
        assert np.allclose(np.linalg.norm(hh - o, axis=1), 0.957)


def test_bead_and_step_displacements():
    reps, _ = inputs.workload("water8_spd_32beads")
    Z, X = reps.stacked()
    base_Z, base_X = inputs.water_cluster_geometry(8, 2)
    dx = (X - base_X[None] * A) / A
    sH = dx[:, Z == 1].std()
    sO = dx[:, Z == 8].std()
    assert abs(sH - 0.1) < 0.01 and abs(sO - 0.03) < 0.004
    seq = inputs.markov_steps(reps, 3, seed=97)
    step = (seq[1].stacked()[1] - X) / A
    assert abs(step[:, Z == 1].std() - 0.1 / np.sqrt(10)) < 0.004


def test_cluster_sets_for_the_learned_guess():
    sets = inputs.water_cluster_set(4, 3, 5, 50)
    assert len(sets) == 3 and all(s.nrep == 5 for s in sets)
    Xs = [s.stacked()[1] for s in sets]
    assert not np.allclose(Xs[0][0], Xs[1][0])
    again = inputs.water_cluster_set(4, 3, 5, 50)
    for a, b in zip(sets, again):
        np.testing.assert_array_equal(a.stacked()[1], b.stacked()[1])


def test_diels_alder_images():
    reps, kind = inputs.workload("da_images_24")
    assert reps.nrep == 24
    nat = [len(z) for z in reps.Z]
    assert nat == [22 + 3 * (i % 5) for i in range(24)]
    for z, x in zip(reps.Z, reps.coords):
        assert (z == 6).sum() == 9 and (z == 8).sum() == 1 + (len(z) - 22) // 3
        d = np.linalg.norm(x[:, None] - x[None], axis=-1)
        np.fill_diagonal(d, np.inf)
        assert d.min() > 0.8 * A
    nbf = [inputs.nbf_of(inputs.basis_set(kind), z) for z in reps.Z]
    assert min(nbf) == 200 and max(nbf) == 296
