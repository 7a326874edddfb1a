"""Pins for the CPU oracle: values that the mathematics or a printed worked
example fixes, independent of the oracle's own formulas.

Every test here is CPU-only. A plausible slip anywhere in the oracle (a dropped
term, a wrong sign or index, a transposed operand) should fail at least one:

* Boys function vs mpmath quadrature and its special values / recursion;
* s-type overlap, kinetic, nuclear-attraction and Coulomb integrals vs their
  closed forms (F_0 via erf);
* p- and d-type integrals vs finite-difference derivatives of the s-type closed
  forms with respect to the centre (d/dA_x e^{-a|r-A|^2} = 2a (x-A_x) e^{..});
* the H2 / STO-3G worked example of Szabo & Ostlund (golden file);
* 8-fold permutational symmetry and positive semi-definiteness of the ERIs;
* unit diagonal of S for normalised contracted (spherical) functions;
* energy invariance under rigid motion, guess and DIIS settings, screening;
* gradient vs central finite differences of the energy, zero net force and
  zero net torque.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1601_02713_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _erf_F0(x):
    return 1.0 if x < 1e-15 else 0.5 * math.sqrt(math.pi / x) * math.erf(math.sqrt(x))


# --------------------------------------------------------------------------- Boys
@pytest.mark.parametrize("m", [0, 1, 2, 3, 5, 8, 10])
def test_boys_vs_mpmath(m):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for T in [0.0, 1e-8, 1e-3, 0.3, 1.0, 2.5, 7.0, 15.0, 29.99, 30.01, 45.0, 120.0]:
        ex = mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, 1])
        v = O.boys(m, T)
        assert abs(v - float(ex)) <= 2e-15 * float(ex), (m, T, v, ex)


def test_boys_special_values_and_recursion():
    for m in range(12):
        assert O.boys(m, 0.0) == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)
    for T in [0.05, 0.7, 3.0, 12.0, 31.0, 60.0]:
        assert O.boys(0, T) == pytest.approx(_erf_F0(T), rel=1e-14)
        for m in range(10):
            lhs = O.boys(m, T)
            rhs = (2 * T * O.boys(m + 1, T) + math.exp(-T)) / (2 * m + 1)
            assert lhs == pytest.approx(rhs, rel=1e-13)


# --------------------------------------------------------- s-type closed forms
def _single_prim_basis(exps, ls):
    """Each 'element' k+1 carries one single-primitive shell (l, a)."""
    return {k + 1: [I.Shell(l, [a], [1.0])] for k, (a, l) in enumerate(zip(exps, ls))}


def test_s_type_closed_forms():
    exps = [0.8, 1.7, 0.35, 2.4]
    Z = np.array([1, 2, 3, 4], np.int32)
    xyz = np.array([[0.1, -0.2, 0.3], [1.1, 0.4, -0.5], [-0.7, 1.3, 0.9], [0.5, -1.2, 1.6]])
    b = _single_prim_basis(exps, [0] * 4)
    ob = O.OracleBasis.build(b, Z, xyz)
    S, T, V = O.one_electron(ob, Z, xyz)
    Nn = [(2 * a / math.pi) ** 0.75 for a in exps]
    for i in range(4):
        for j in range(4):
            a, bb = exps[i], exps[j]
            p, mu = a + bb, a * bb / (a + bb)
            R2 = float(np.sum((xyz[i] - xyz[j]) ** 2))
            s = Nn[i] * Nn[j] * (math.pi / p) ** 1.5 * math.exp(-mu * R2)
            assert S[i, j] == pytest.approx(s, rel=1e-13)
            assert T[i, j] == pytest.approx(mu * (3 - 2 * mu * R2) * s, rel=1e-12)
            P = (a * xyz[i] + bb * xyz[j]) / p
            v = 0.0
            for c in range(4):
                RPC2 = float(np.sum((P - xyz[c]) ** 2))
                v += -Z[c] * 2 * math.pi / p * Nn[i] * Nn[j] * math.exp(-mu * R2) * _erf_F0(p * RPC2)
            assert V[i, j] == pytest.approx(v, rel=1e-12)
    eri = O.eri_full(ob)
    for (i, j, k, l) in [(0, 0, 0, 0), (0, 1, 2, 3), (3, 2, 1, 0), (1, 1, 2, 2), (0, 3, 0, 3), (2, 1, 3, 3)]:
        a, bb, c, d = exps[i], exps[j], exps[k], exps[l]
        p, q = a + bb, c + d
        P = (a * xyz[i] + bb * xyz[j]) / p
        Q = (c * xyz[k] + d * xyz[l]) / q
        Kab = math.exp(-a * bb / p * float(np.sum((xyz[i] - xyz[j]) ** 2)))
        Kcd = math.exp(-c * d / q * float(np.sum((xyz[k] - xyz[l]) ** 2)))
        rho = p * q / (p + q)
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * _erf_F0(rho * float(np.sum((P - Q) ** 2)))
        ref *= Nn[i] * Nn[j] * Nn[k] * Nn[l]
        assert eri[i, j, k, l] == pytest.approx(ref, rel=1e-12)


# ------------------------------------------- p and d via derivatives of s forms
def _eri_ssss_unnorm(a, A, b, B, c, C, d, D):
    p, q = a + b, c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    Kab = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
    Kcd = math.exp(-c * d / q * float(np.sum((C - D) ** 2)))
    rho = p * q / (p + q)
    return 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * _erf_F0(rho * float(np.sum((P - Q) ** 2)))


def _ovl_unnorm(a, A, b, B):
    p = a + b
    return (math.pi / p) ** 1.5 * math.exp(-a * b / p * float(np.sum((A - B) ** 2)))


def test_p_and_d_integrals_from_centre_derivatives():
    a, b, c, d = 0.9, 1.3, 0.6, 2.1
    xyz = np.array([[0.2, -0.1, 0.4], [1.0, 0.5, -0.3], [-0.6, 0.9, 0.7], [0.4, -0.8, 1.1]])
    Z = np.array([1, 2, 3, 4], np.int32)
    # atom 0: p shell; atom 1: d shell; atoms 2, 3: s shells
    bas = {1: [I.Shell(1, [a], [1.0])], 2: [I.Shell(2, [b], [1.0])],
           3: [I.Shell(0, [c], [1.0])], 4: [I.Shell(0, [d], [1.0])]}
    ob = O.OracleBasis.build(bas, Z, xyz)
    Np = (2 * a / math.pi) ** 0.75 * math.sqrt(4 * a)              # x^1 normalisation
    Nd = (2 * b / math.pi) ** 0.75 * (4 * b) / math.sqrt(3.0)       # x^2 normalisation
    Ns = [(2 * e / math.pi) ** 0.75 for e in (c, d)]
    h = 1e-4
    A, B, C, D = xyz

    def dA(f, x, *args):  # d/dA_x of f(A, ...) by central differences
        e = np.zeros(3)
        e[x] = h
        return (f(A + e, *args) - f(A - e, *args)) / (2 * h)

    # (p_x s | s s): basis function index 0..2 = p_x, p_y, p_z on atom 0
    blk = O.eri_block(ob, 0, 2, 2, 3)  # (p s_c | s_c s_d)
    for x in range(3):
        ref = Np * Ns[0] * Ns[0] * Ns[1] / (2 * a) * dA(lambda AA: _eri_ssss_unnorm(a, AA, c, C, c, C, d, D), x)
        assert blk[x, 0, 0, 0] == pytest.approx(ref, rel=2e-8, abs=1e-12)
    # overlap <p_x | s_d>
    S, _, _ = O.one_electron(ob, Z, xyz)
    ip0, is_d = 0, 3 + 5 + 1  # p(3) + d(5) + s_c(1) -> s_d index 9
    for x in range(3):
        ref = Np * Ns[1] / (2 * a) * dA(lambda AA: _ovl_unnorm(a, AA, d, D), x)
        assert S[ip0 + x, is_d] == pytest.approx(ref, rel=2e-8, abs=1e-12)
    # d functions: sqrt3 xy (m=-2) and zz - (xx+yy)/2 (m=0) on atom 1 vs second derivatives

    def d2B(f, x, y):
        ex = np.zeros(3)
        ey = np.zeros(3)
        ex[x] = h
        ey[y] = h
        return (f(B + ex + ey) - f(B + ex - ey) - f(B - ex + ey) + f(B - ex - ey)) / (4 * h * h)

    f_ov = lambda BB: _ovl_unnorm(b, BB, c, C)  # noqa: E731
    cart = {}
    for (x, y) in [(0, 1), (0, 0), (1, 1), (2, 2)]:
        dd = d2B(f_ov, x, y)
        if x == y:  # (x-B)^2 g = [d2/dB^2 g + 2b g] / (4 b^2)
            dd += 2 * b * f_ov(B)
        cart[(x, y)] = dd / (4 * b * b)
    is_c = 3 + 5
    assert S[3 + 0, is_c] == pytest.approx(Nd * Ns[0] * math.sqrt(3) * cart[(0, 1)], rel=1e-6, abs=1e-10)
    ref0 = Nd * Ns[0] * (cart[(2, 2)] - 0.5 * (cart[(0, 0)] + cart[(1, 1)]))
    assert S[3 + 2, is_c] == pytest.approx(ref0, rel=1e-6, abs=1e-10)


# ------------------------------------------------------------ worked example
def test_h2_sto3g_textbook():
    g = json.load(open(os.path.join(GOLDEN, "h2_sto3g.json")))
    z = g["zeta"]
    bas = {1: [I.Shell(0, [e * z * z for e in g["sto3g_zeta1_exponents"]], g["sto3g_coefficients"])]}
    Z = np.array([1, 1], np.int32)
    xyz = np.array([[0, 0, 0], [0, 0, g["R_bohr"]]], float)
    ob = O.OracleBasis.build(bas, Z, xyz)
    S, T, V = O.one_electron(ob, Z, xyz)
    eri = O.eri_full(ob)
    pr, tol = g["printed"], g["tolerance"]
    got = {"S12": S[0, 1], "T11": T[0, 0], "T12": T[0, 1], "V11_total": V[0, 0], "V12_total": V[0, 1],
           "eri_1111": eri[0, 0, 0, 0], "eri_1122": eri[0, 0, 1, 1], "eri_2111": eri[1, 0, 0, 0],
           "eri_2121": eri[1, 0, 1, 0]}
    E, _, res = O.rhf_energy_gradient(bas, Z, xyz, want_gradient=False)
    got["E_total"] = E
    got["E_electronic"] = E - res.e_nn
    for k, v in pr.items():
        assert abs(got[k] - v) <= tol, (k, got[k], v)


# ------------------------------------------------------------- ERI structure
@pytest.fixture(scope="module")
def water_spd():
    b = I.basis_set("split_spd")
    Z, xyz = I.small_molecule("water")
    return b, Z, xyz, O.OracleBasis.build(b, Z, xyz)


def test_eri_eightfold_symmetry_and_psd(water_spd):
    b, Z, xyz, ob = water_spd
    g = O.eri_full(ob)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0), (2, 3, 1, 0)]:
        np.testing.assert_allclose(g, g.transpose(perm), rtol=0, atol=1e-13)
    N = ob.nbf
    w = np.linalg.eigvalsh(g.reshape(N * N, N * N))
    assert w.min() > -1e-12 * w.max()


def test_overlap_unit_diagonal(water_spd):
    b, Z, xyz, ob = water_spd
    S, T, V = O.one_electron(ob, Z, xyz)
    np.testing.assert_allclose(np.diag(S), 1.0, atol=1e-13)
    np.testing.assert_allclose(S, S.T, atol=1e-15)
    np.testing.assert_allclose(T, T.T, atol=1e-13)
    np.testing.assert_allclose(V, V.T, atol=1e-12)


def test_jk_matches_full_tensor(water_spd):
    b, Z, xyz, ob = water_spd
    g = O.eri_full(ob)
    rng = np.random.default_rng(5)
    D = rng.normal(size=(ob.nbf, ob.nbf))
    D = D + D.T
    J, K, _ = O.jk(ob, D, 0.0)
    np.testing.assert_allclose(J, np.einsum("mnls,ls->mn", g, D), atol=1e-11)
    np.testing.assert_allclose(K, np.einsum("mlns,ls->mn", g, D), atol=1e-11)


@pytest.mark.parametrize("system", ["water", "dimer"])
def test_g_block_matches_jk(water_spd, system):
    """Every shell-pair block of the oracle's sampled Fock-block routine
    (g_block: G = J - K/2 summed over every ordered shell pair, no screening)
    equals J - K/2 from the canonical-quartet J/K routine, which is itself
    pinned to the full ERI tensor above. A transposed K index, a missing 1/2
    or a dropped permutation in g_block fails here. Water and the water dimer
    in the s/p/d basis (d-d, d-p and cross-molecule blocks)."""
    b = water_spd[0]
    if system == "water":
        Z, xyz, ob = water_spd[1], water_spd[2], water_spd[3]
    else:
        r, _ = I.workload("water2_min_4beads")
        Z, c = r.stacked()
        xyz = c[0]
        ob = O.OracleBasis.build(b, Z, xyz)
    N = ob.nbf
    rng = np.random.default_rng(11)
    D = rng.normal(size=(N, N))
    D = D + D.T
    J, K, _ = O.jk(ob, D, 0.0)
    G = J - 0.5 * K
    off = np.cumsum([0] + [ob.shell_nbf(s) for s in range(len(ob.l))])
    scale = np.abs(G).max()
    for a in range(len(ob.l)):
        for bb in range(len(ob.l)):
            blk = O.g_block(ob, D, a, bb)
            ref = G[off[a]:off[a + 1], off[bb]:off[bb + 1]]
            assert np.abs(blk - ref).max() <= 1e-12 * scale, (system, a, bb)


# ---------------------------------------------------------------- full RHF
def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


@pytest.fixture(scope="module")
def dimer_min():
    r, kind = I.workload("water2_min_4beads")
    Z, c = r.stacked()
    b = I.basis_set(kind)
    E, g, res = O.rhf_energy_gradient(b, Z, c[0])
    return b, Z, c[0], E, g, res


def test_energy_rigid_motion_invariance(dimer_min):
    b, Z, xyz, E, g, res = dimer_min
    R = _rot([0.3, -1.0, 0.5], 0.77)
    E2 = O.rhf_energy_gradient(b, Z, xyz @ R.T + np.array([1.5, -0.4, 2.2]), want_gradient=False)[0]
    assert abs(E2 - E) < 1e-10


def test_energy_independent_of_guess_and_diis(dimer_min):
    b, Z, xyz, E, g, res = dimer_min
    ob = O.OracleBasis.build(b, Z, xyz)
    r2 = O.run_scf(ob, Z, xyz, diis_size=4)
    assert abs(r2.energy - E) < 1e-10
    N = ob.nbf
    D0 = res.D + 0.02 * np.random.default_rng(3).normal(size=(N, N))
    r3 = O.run_scf(ob, Z, xyz, D0=(D0 + D0.T) / 2)
    assert abs(r3.energy - E) < 1e-10


def test_screening_changes_energy_below_1e9(dimer_min):
    b, Z, xyz, E, g, res = dimer_min
    E0 = O.rhf_energy_gradient(b, Z, xyz, want_gradient=False, tau=0.0)[0]
    assert abs(E0 - E) < 1e-9


def test_gradient_invariances(dimer_min):
    b, Z, xyz, E, g, res = dimer_min
    assert np.abs(g.sum(0)).max() < 1e-9
    torque = np.cross(xyz, g).sum(0)
    assert np.abs(torque).max() < 1e-8


def test_gradient_vs_finite_differences(dimer_min):
    b, Z, xyz, E, g, res = dimer_min
    h = 1e-4
    for (a, x) in [(0, 0), (1, 2), (2, 1), (4, 0), (5, 2)]:
        xp = xyz.copy()
        xp[a, x] += h
        xm = xyz.copy()
        xm[a, x] -= h
        Ep = O.rhf_energy_gradient(b, Z, xp, want_gradient=False)[0]
        Em = O.rhf_energy_gradient(b, Z, xm, want_gradient=False)[0]
        assert abs((Ep - Em) / (2 * h) - g[a, x]) < 5e-8


def test_gradient_fd_with_d_functions(water_spd):
    b, Z, xyz, ob = water_spd
    E, g, res = O.rhf_energy_gradient(b, Z, xyz)
    assert res.converged
    h = 1e-4
    for (a, x) in [(0, 2), (1, 0), (2, 2)]:
        xp = xyz.copy()
        xp[a, x] += h
        xm = xyz.copy()
        xm[a, x] -= h
        Ep = O.rhf_energy_gradient(b, Z, xp, want_gradient=False)[0]
        Em = O.rhf_energy_gradient(b, Z, xm, want_gradient=False)[0]
        assert abs((Ep - Em) / (2 * h) - g[a, x]) < 5e-8
