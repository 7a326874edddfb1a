"""Pins of the learned-guess oracle (oracle/guess.py), CPU only: the local
pair frames and block rotations make converged density blocks invariant
under a rigid motion of the molecule; the features are invariant; the shell
representations are orthogonal and multiplicative; the MLP gradient matches
central finite differences."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import guess as GO
from paper_1601_02713_gb300 import inputs as I


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_shell_representation_orthogonal_and_multiplicative():
    U1, U2 = _rot([1, 2, 3], 0.7), _rot([-2, 0.5, 1], 1.9)
    for l in (0, 1, 2):
        M1, M2, M12 = GO.shell_rotation(l, U1), GO.shell_rotation(l, U2), GO.shell_rotation(l, U2 @ U1)
        n = M1.shape[0]
        np.testing.assert_allclose(M1.T @ M1, np.eye(n), atol=1e-13)
        # phi_lab = M(U) phi_local: composing frames composes the matrices
        np.testing.assert_allclose(M12, M1 @ M2, atol=1e-13)


def _blocks_local(bas, Z, xyz, D):
    ob = O.OracleBasis.build(bas, Z, xyz)
    # functions of each atom are contiguous (shells listed atom by atom)
    per_atom = {}
    o = 0
    for s in range(len(ob.l)):
        a = int(ob.atom[s])
        n = ob.shell_nbf(s)
        per_atom.setdefault(a, [o, o, []])
        per_atom[a][1] = o + n
        per_atom[a][2].append(int(ob.l[s]))
        o += n
    out = {}
    for A in range(len(Z)):
        for B in range(A, len(Z)):
            U = GO.pair_frame(xyz, A, B)
            a0, a1, la = per_atom[A]
            b0, b1, lb = per_atom[B]
            out[(A, B)] = GO.to_local(D[a0:a1, b0:b1], GO.atom_rotation(la, U), GO.atom_rotation(lb, U))
    return out


def test_local_blocks_invariant_under_rigid_motion():
    bas = I.basis_set("split_spd")
    Z, xyz = I.small_molecule("water")
    xyz = xyz + np.array([[0.05, -0.02, 0.03], [0.0, 0.04, -0.1], [0.02, 0.0, 0.07]])  # break symmetry
    E1, _, r1 = O.rhf_energy_gradient(bas, Z, xyz, want_gradient=False)
    Q = _rot([0.3, -1.0, 0.4], 2.1)
    xyz2 = xyz @ Q.T + np.array([0.7, -1.3, 2.0])
    E2, _, r2 = O.rhf_energy_gradient(bas, Z, xyz2, want_gradient=False)
    assert abs(E1 - E2) < 1e-9
    b1 = _blocks_local(bas, Z, xyz, r1.D)
    b2 = _blocks_local(bas, Z, xyz2, r2.D)
    for k in b1:
        np.testing.assert_allclose(b2[k], b1[k], atol=2e-7)


def test_features_invariant_under_rigid_motion():
    r, _ = I.workload("water8_spd_32beads", nrep=1)
    Z, X = r.stacked()
    xyz = X[0]
    Q = _rot([1, 1, -2], 0.9)
    xyz2 = xyz @ Q.T + 3.0
    for (A, B) in [(0, 0), (0, 1), (3, 17), (12, 12)]:
        np.testing.assert_allclose(GO.pair_features(Z, xyz2, A, B), GO.pair_features(Z, xyz, A, B), atol=1e-10)


def test_mlp_gradient_vs_finite_differences():
    rng = np.random.default_rng(4)
    dims = [12, 16, 16, 7]
    params = [(rng.normal(size=(a, b)) / math.sqrt(a), rng.normal(size=b) * 0.1) for a, b in zip(dims[:-1], dims[1:])]
    X = rng.normal(size=(9, dims[0]))
    Y = rng.normal(size=(9, dims[-1]))
    L, grads = GO.mse_loss_and_grads(params, X, Y)
    h = 1e-6
    for k in range(len(params)):
        W, b = params[k]
        for (i, j) in [(0, 0), (3, 5), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = W.copy()
            Wp[i, j] += h
            Wm = W.copy()
            Wm[i, j] -= h
            Lp = GO.mse_loss_and_grads(params[:k] + [(Wp, b)] + params[k + 1:], X, Y)[0]
            Lm = GO.mse_loss_and_grads(params[:k] + [(Wm, b)] + params[k + 1:], X, Y)[0]
            assert abs((Lp - Lm) / (2 * h) - grads[k][0][i, j]) < 1e-7
        bp = b.copy()
        bp[1] += h
        bm = b.copy()
        bm[1] -= h
        Lp = GO.mse_loss_and_grads(params[:k] + [(W, bp)] + params[k + 1:], X, Y)[0]
        Lm = GO.mse_loss_and_grads(params[:k] + [(W, bm)] + params[k + 1:], X, Y)[0]
        assert abs((Lp - Lm) / (2 * h) - grads[k][1][1]) < 1e-7


def test_frames_of_degenerate_geometries():
    """Frames stay orthonormal and right-handed when the reference atom lies
    on the pair axis (a linear molecule) and when there is no third atom."""
    cases = [np.array([[0.0, 0, 0], [0, 0, 1.8], [0, 0, 3.6]]),   # O-H-H on a line
             np.array([[0.0, 0, 0], [0, 0, 1.4]]),                # H2
             np.array([[0.0, 0, 0], [1.8, 0, 0], [3.6, 0, 0]])]   # along x: e_z nearly x
    for xyz in cases:
        n = len(xyz)
        for A in range(n):
            for B in range(n):
                U = GO.pair_frame(xyz, A, B)
                np.testing.assert_allclose(U @ U.T, np.eye(3), atol=1e-12)
                assert abs(np.linalg.det(U) - 1.0) < 1e-12
                if A != B:
                    ez = (xyz[B] - xyz[A]) / np.linalg.norm(xyz[B] - xyz[A])
                    np.testing.assert_allclose(U[2], ez, atol=1e-12)
