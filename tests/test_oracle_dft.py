"""Pins of the B3LYP oracle (`oracle/dft.py`) against what the mathematics
fixes, not against itself: the grid's integrals of the oracle's own analytic
overlap and electron count, the basis derivatives against finite
differences, the hydrogen atom's local and B88 exchange energies, the
uniform-scaling law of the exchange functionals, the
equality of the two published forms of LYP, LYP's zero for a one-spin
density and its uniform-density limit, VWN's exact high-density coefficient
and the uniform-gas correlation energies VWN5 was fitted to, the Kohn-Sham matrix as the
derivative of the energy, the reduction to RHF at full exact exchange, and
the analytic gradient against central finite differences of the energy."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import dft
from paper_1601_02713_gb300 import inputs

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def water():
    bas = inputs.basis_set("split_spd")
    Z, X = inputs.small_molecule("water")
    ob = O.OracleBasis.build(bas, Z, X)
    pts, w = dft.molecular_grid(X)
    phi, g, lap = dft.ao_values(ob, pts, laplacian=True)
    scf = O.run_scf(ob, Z, X)
    return dict(bas=bas, Z=Z, X=X, ob=ob, pts=pts, w=w, phi=phi, g=g, lap=lap, D=scf.D, S=scf.S, E_rhf=scf.energy)


def test_grid_integrates_the_overlap_and_the_electrons(water):
    """INT phi_m phi_n on the Becke grid = the oracle's analytic overlap
    (McMurchie-Davidson); INT rho = tr(D S) = N."""
    phi, w = water["phi"], water["w"]
    Sg = (phi * w[:, None]).T @ phi
    assert np.abs(Sg - water["S"]).max() < 2e-6
    rho, _, _ = dft.density_on_grid(water["D"], phi, water["g"])
    assert abs(float(np.sum(w * rho)) - 10.0) < 1e-6


def test_basis_derivatives_against_finite_differences(water):
    ob = water["ob"]
    rng = np.random.default_rng(5)
    p = water["X"][rng.integers(0, 3, 12)] + rng.normal(scale=0.6, size=(12, 3))
    phi, g, lap = dft.ao_values(ob, p, laplacian=True)
    h = 1e-4
    num_g = np.zeros_like(g)
    num_l = np.zeros_like(lap)
    for x in range(3):
        e = np.zeros(3)
        e[x] = h
        fp, _, _ = dft.ao_values(ob, p + e)
        fm, _, _ = dft.ao_values(ob, p - e)
        num_g[x] = (fp - fm) / (2 * h)
        num_l += (fp - 2 * phi + fm) / h ** 2
    scale = np.abs(phi).max()
    assert np.abs(num_g - g).max() < 1e-6 * scale * 100
    assert np.abs(num_l - lap).max() < 1e-3 * np.abs(lap).max()


def test_exchange_scales_uniformly(water):
    """E_x[rho_l] = l E_x[rho] for rho_l(r) = l^3 rho(l r) (exact for
    exchange; Levy and Perdew): the molecule shrunk by l with exponents
    times l^2 and the same density matrix has exactly rho_l, and the grid
    scaled alongside integrates it with the same quadrature."""
    lam = 1.37
    bas = {z: [inputs.Shell(s.l, [a * lam ** 2 for a in s.exps], s.coefs) for s in shells]
           for z, shells in water["bas"].items()}
    X2 = water["X"] / lam
    ob2 = O.OracleBasis.build(bas, water["Z"], X2)
    pts2, w2 = dft.molecular_grid(X2, Rm=1.0 / lam)
    phi2, g2, _ = dft.ao_values(ob2, pts2)
    D = water["D"]
    for f in (lambda r, s: dft.lda_x(r), lambda r, s: dft.lda_x(r) + dft.b88_dx(r, s)):
        E1, _ = dft.xc_energy_matrix(D, water["phi"], water["g"], water["w"], f)
        E2, _ = dft.xc_energy_matrix(D, phi2, g2, w2, f)
        assert E1 < 0
        assert abs(E2 - lam * E1) < 1e-9 * abs(E1)
    # correlation has no such law: LYP does not scale linearly
    E1, _ = dft.xc_energy_matrix(D, water["phi"], water["g"], water["w"], dft.lyp)
    E2, _ = dft.xc_energy_matrix(D, phi2, g2, w2, dft.lyp)
    assert abs(E2 - lam * E1) > 1e-3 * abs(E1)


def test_the_two_forms_of_lyp_have_the_same_integral(water):
    """Miehlich et al.'s form is LYP's 1988 form with the Laplacian terms
    integrated by parts: pointwise different, equal integrals."""
    rho, grho, lrho = dft.density_on_grid(water["D"], water["phi"], water["g"], water["lap"])
    keep = rho > 1e-10
    r = torch.tensor(rho[keep], dtype=torch.float64)
    s = torch.tensor(np.sum(grho[:, keep] ** 2, axis=0), dtype=torch.float64)
    lp = torch.tensor(lrho[keep], dtype=torch.float64)
    w = water["w"][keep]
    e_m = dft.lyp(r, s).numpy()
    e_o = dft.lyp_original(r, s, lp).numpy()
    Em, Eo = float(np.sum(w * e_m)), float(np.sum(w * e_o))
    assert Em < 0
    assert abs(Em - Eo) < 2e-5 * abs(Em), (Em, Eo)
    assert np.abs(e_m - e_o).max() > 1e-3 * np.abs(e_m).max()   # pointwise they differ


def test_lyp_vanishes_for_a_one_spin_density():
    """LYP has no self-interaction for one-electron (fully polarised)
    densities: E_c = 0 whenever rho_b = 0."""
    rng = np.random.default_rng(7)
    ra = torch.tensor(rng.uniform(1e-3, 5.0, 50), dtype=torch.float64)
    gaa = torch.tensor(rng.uniform(0.0, 10.0, 50), dtype=torch.float64)
    z = torch.zeros(50, dtype=torch.float64)
    e = dft.lyp_spin(ra, z, gaa, z, z).numpy()
    assert np.abs(e).max() < 1e-15 * float(ra.max()) ** 2


def test_lyp_uniform_limit():
    """For a uniform closed-shell density both forms reduce pointwise to
    -a rho (1 + b C_F exp(-c rho^{-1/3})) / (1 + d rho^{-1/3}), which is negative."""
    r = torch.tensor(np.geomspace(1e-4, 1e3, 40), dtype=torch.float64)
    z = torch.zeros_like(r)
    a, b, c, d = dft.LYP_A, dft.LYP_B, dft.LYP_C, dft.LYP_D
    CF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)
    ref = (-a * r * (1.0 + b * CF * torch.exp(-c * r ** (-1.0 / 3.0))) / (1.0 + d * r ** (-1.0 / 3.0))).numpy()
    for e in (dft.lyp(r, z).numpy(), dft.lyp_original(r, z, z).numpy()):
        np.testing.assert_allclose(e, ref, rtol=1e-13, atol=0)
    assert ref.max() < 0


@pytest.mark.parametrize("kind", ["rpa", "5"])
def test_vwn_high_density_coefficient(kind):
    """Both VWN fits keep the exact high-density behaviour eps_c ~ A ln rs
    with A = (1 - ln 2) / pi^2 (Gell-Mann and Brueckner)."""
    r1 = torch.tensor([1e-9], dtype=torch.float64)
    r2 = torch.tensor([1e-8], dtype=torch.float64)
    slope = float(dft.vwn_eps(r2, kind) - dft.vwn_eps(r1, kind)) / math.log(10.0)
    assert abs(slope - (1.0 - math.log(2.0)) / math.pi ** 2) < 2e-4
    # correlation lowers the energy at metallic densities
    assert float(dft.vwn_eps(torch.tensor([2.0], dtype=torch.float64), kind)) < 0


def test_hydrogen_atom_exchange():
    """Exchange energies of the hydrogen atom's exact density e^{-2r}/pi (one
    spin; closed-shell functional on twice the density, halved: the spin
    scaling of exchange): the local (Dirac-Slater) value in closed form,
    -(3/2)(3/(4 pi))^{1/3} (27/64) pi^{-1/3} = -0.26804, and Becke's 1988
    value for B88, -0.3098 hartree (exact: -0.3125)."""
    pts, w = dft.molecular_grid(np.zeros((1, 3)), n_rad=200, n_theta=8)
    r = np.linalg.norm(pts, axis=1)
    rho_a = np.exp(-2.0 * r) / math.pi
    keep = rho_a > 1e-14
    rho_a, w = rho_a[keep], w[keep]
    rho = torch.tensor(2.0 * rho_a, dtype=torch.float64)
    sigma = torch.tensor((2.0 * 2.0 * rho_a) ** 2, dtype=torch.float64)   # |d rho/dr| = 2 rho
    e_lda = 0.5 * float(np.sum(w * dft.lda_x(rho).numpy()))
    e_b88 = 0.5 * float(np.sum(w * (dft.lda_x(rho) + dft.b88_dx(rho, sigma)).numpy()))
    closed = -1.5 * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0) * 27.0 / 64.0 * math.pi ** (-1.0 / 3.0)
    assert abs(e_lda - closed) < 1e-9
    assert abs(e_b88 - (-0.3098)) < 2e-4


def test_vwn5_reproduces_the_uniform_gas_correlation():
    """VWN's recommended fit reproduces the Ceperley-Alder quantum Monte Carlo
    correlation energies of the unpolarised uniform gas it was fitted to
    (hartree per electron; the Perdew-Wang 1992 tabulation of the same
    data): -0.0600, -0.0448, -0.0281, -0.0185 at rs = 1, 2, 5, 10. The RPA fit
    lies below them (RPA overestimates correlation)."""
    for rs, ref in ((1.0, -0.0600), (2.0, -0.0448), (5.0, -0.0281), (10.0, -0.0185)):
        t = torch.tensor([rs], dtype=torch.float64)
        assert abs(float(dft.vwn_eps(t, "5")) - ref) < 3e-4, rs
        assert float(dft.vwn_eps(t, "rpa")) < ref - 0.005


def test_b88_is_local_exchange_without_a_gradient():
    r = torch.tensor([0.01, 0.3, 2.0], dtype=torch.float64)
    assert float(torch.abs(dft.b88_dx(r, torch.zeros(3, dtype=torch.float64))).max()) == 0.0
    assert float(dft.b88_dx(r, torch.ones(3, dtype=torch.float64)).max()) < 0


def test_ks_matrix_is_the_derivative_of_the_energy(water):
    """V_mn = dE_xc / dD_mn (symmetric perturbation), the GGA terms included."""
    D, phi, g, w = water["D"], water["phi"], water["g"], water["w"]
    E0, V = dft.xc_energy_matrix(D, phi, g, w)
    rng = np.random.default_rng(3)
    P = rng.normal(size=D.shape)
    P = 0.5 * (P + P.T)
    eps = 1e-5
    Ep, _ = dft.xc_energy_matrix(D + eps * P, phi, g, w)
    Em, _ = dft.xc_energy_matrix(D - eps * P, phi, g, w)
    assert abs((Ep - Em) / (2 * eps) - float(np.sum(V * P))) < 1e-6 * abs(float(np.sum(V * P)))


def test_blocked_grid_sums_equal_the_whole(water):
    D, w, pts = water["D"], water["w"], water["pts"]
    E0, V0 = dft.xc_energy_matrix(D, water["phi"], water["g"], w)
    E1, V1 = dft.xc_on_grid(water["ob"], D, pts, w, chunk=7919)
    assert abs(E1 - E0) < 1e-11 * abs(E0)
    assert np.abs(V1 - V0).max() < 1e-11 * np.abs(V0).max()


def test_full_exact_exchange_without_xc_is_rhf(water):
    res = dft.ks_scf(water["ob"], water["Z"], water["X"], func=None, a0=1.0)
    assert res["converged"]
    assert abs(res["energy"] - water["E_rhf"]) < 1e-9


def test_b3lyp_scf_converges_on_a_converged_grid(water):
    """The B3LYP SCF converges, its energy lies below RHF's (the
    correlation), and a finer grid moves it by less than 1e-5 hartree."""
    res = dft.ks_scf(water["ob"], water["Z"], water["X"], grid=(water["pts"], water["w"]))
    assert res["converged"]
    assert res["energy"] < water["E_rhf"] - 0.1
    fine = dft.molecular_grid(water["X"], n_rad=90, n_theta=22)
    res2 = dft.ks_scf(water["ob"], water["Z"], water["X"], grid=fine)
    assert abs(res2["energy"] - res["energy"]) < 1e-5


def _distorted_water():
    Z, X = inputs.small_molecule("water")
    return Z, X + np.random.default_rng(11).normal(scale=0.05, size=X.shape)


COORDS = [(0, 2), (1, 1), (2, 0)]


def test_exact_exchange_fraction_in_the_gradient():
    """A hybrid without an XC term (F = h + J - kx K/2) pins the two-electron
    gradient's exact-exchange fraction kx against central differences."""
    bas = inputs.basis_set("split_spd")
    Z, X = _distorted_water()
    kx = 0.5
    ob = O.OracleBasis.build(bas, Z, X)
    res = dft.ks_scf(ob, Z, X, func=None, a0=kx, conv_energy=1e-12, conv_error=1e-10)
    g = (O.grad_1e(ob, Z, X, res["D"], res["W"]) + O.grad_2e(ob, len(Z), res["D"], kx=kx)
         + O.nuclear_repulsion(Z, X)[1])
    h = 1e-4
    for a, x in COORDS:
        E = []
        for sgn in (1, -1):
            Xs = X.copy()
            Xs[a, x] += sgn * h
            E.append(dft.ks_scf(O.OracleBasis.build(bas, Z, Xs), Z, Xs, func=None, a0=kx,
                                conv_energy=1e-12, conv_error=1e-10)["energy"])
        assert abs((E[0] - E[1]) / (2 * h) - g[a, x]) < 2e-7, (a, x)
    # kx = 1 is the Hartree-Fock gradient itself
    np.testing.assert_allclose(O.grad_2e(ob, len(Z), res["D"], kx=1.0), O.grad_2e(ob, len(Z), res["D"]),
                               rtol=0, atol=1e-14)


def test_b3lyp_gradient_against_finite_differences():
    """The B3LYP gradient (one-electron terms with the Kohn-Sham W, 20% exact
    exchange, the XC terms through the basis functions, V_nn) is the
    derivative of the energy on a grid fixed in space."""
    bas = inputs.basis_set("split_spd")
    Z, X = _distorted_water()
    grid = dft.molecular_grid(X, n_rad=50, n_theta=14)
    E0, g, res = dft.b3lyp_energy_gradient(bas, Z, X, grid=grid, conv_energy=1e-12, conv_error=1e-10)
    assert res["converged"]
    h = 1e-4
    for a, x in COORDS:
        E = []
        for sgn in (1, -1):
            Xs = X.copy()
            Xs[a, x] += sgn * h
            E.append(dft.ks_scf(O.OracleBasis.build(bas, Z, Xs), Z, Xs, grid=grid, conv_energy=1e-12,
                                conv_error=1e-10)["energy"])
        assert abs((E[0] - E[1]) / (2 * h) - g[a, x]) < 2e-7, (a, x, (E[0] - E[1]) / (2 * h), g[a, x])
