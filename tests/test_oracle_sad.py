"""Pins of the oracle's spherically averaged atomic density (the building
block of the superposition-of-atomic-densities guess).

* electron count: tr(D S) = Z;
* spherical symmetry: D is unchanged by any rotation of the atom,
  M D M^T = D with M the representation of the rotation on the atom's shells;
* self-consistency: D is built from eigenvectors of F(D), so the commutator
  X^T (F D S - S D F) X vanishes;
* closed shell: for neon (1s^2 2s^2 2p^6) it is the ordinary RHF density.
"""
import numpy as np
import pytest

import oracle as O
from oracle import guess as OG
from paper_1601_02713_gb300 import inputs


def _rot(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def _one_atom(bas, Z):
    Zs = np.array([Z], np.int32)
    xyz = np.zeros((1, 3))
    ob = O.OracleBasis.build(bas, Zs, xyz)
    S, T, V = O.one_electron(ob, Zs, xyz)
    return ob, S, T + V


@pytest.mark.parametrize("kind,Z", [("split_spd", 8), ("split_spd", 6), ("split_spd", 1), ("min_sp", 8)])
def test_sad_density_pins(kind, Z):
    bas = inputs.basis_set(kind)
    D = O.sad_atomic_density(bas, Z)
    ob, S, h = _one_atom(bas, Z)
    assert abs(np.trace(D @ S) - Z) < 1e-10
    np.testing.assert_allclose(D, D.T, atol=1e-14)
    ls = [sh.l for sh in bas[Z]]
    for seed in range(3):
        M = OG.atom_rotation(ls, _rot(seed))
        np.testing.assert_allclose(M @ D @ M.T, D, atol=1e-10)
    J, K, _ = O.jk(ob, D)
    F = h + J - 0.5 * K
    X = O.orthogonaliser(S)
    assert np.abs(X.T @ (F @ D @ S - S @ D @ F) @ X).max() < 1e-7


def test_sad_closed_shell_is_rhf():
    bas = {10: inputs.basis_set("split_spd")[8]}
    D = O.sad_atomic_density(bas, 10)
    Zs = np.array([10], np.int32)
    res = O.run_scf(O.OracleBasis.build(bas, Zs, np.zeros((1, 3))), Zs, np.zeros((1, 3)))
    assert res.converged
    np.testing.assert_allclose(D, res.D, atol=1e-7)


def test_sad_rejects_missing_p_shell():
    bas = {8: [sh for sh in inputs.basis_set("split_spd")[8] if sh.l == 0]}
    with pytest.raises(ValueError):
        O.sad_atomic_density(bas, 8)
