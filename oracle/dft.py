"""Oracle: closed-shell B3LYP Kohn-Sham energy and Fock matrix on a numerical
grid (CPU, FP64).

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: only `tests/` may
import it. It shares no code with the CUDA library.

The paper's level of theory is B3LYP (Sec. 3.1 for the water clusters, Sec.
3.2 for the Diels-Alder string); the GPU path of this project is RHF. This
module is the plain definition of the B3LYP energy and Kohn-Sham matrix of a
closed-shell molecule in the oracle's basis, integrals and SCF conventions
(`rhf.py`), the functionals written from their defining papers:

* B3LYP (Becke's three-parameter hybrid with the LYP correlation):
    E_xc = 0.08 E_x^LDA + 0.72 E_x^B88 + 0.20 E_x^HF + 0.19 E_c^VWN + 0.81 E_c^LYP,
  E_x^B88 being Becke's 1988 exchange including its local part, so that the
  local exchange carries 0.80 and the gradient correction 0.72.
* LDA exchange (Dirac-Slater), closed shell: e_x = -(3/4) (3/pi)^{1/3} rho^{4/3}.
* B88 gradient correction (Becke 1988), per spin:
    -beta rho_s^{4/3} x_s^2 / (1 + 6 beta x_s asinh x_s), x_s = |grad rho_s| / rho_s^{4/3},
  beta = 0.0042; closed shell: rho_s = rho / 2, |grad rho_s| = |grad rho| / 2.
* VWN correlation (Vosko, Wilk, Nusair 1980), paramagnetic interpolation
    eps_c = A [ ln(x^2/X(x)) + (2b/Q) atan(Q/(2x+b))
                - (b x0 / X(x0)) ( ln((x-x0)^2/X(x)) + (2(b+2x0)/Q) atan(Q/(2x+b)) ) ],
  x = sqrt(rs), X(x) = x^2 + b x + c, Q = sqrt(4c - b^2), rs = (3/(4 pi rho))^{1/3},
  A = 0.0310907. Reading: B3LYP as the hybrid is used in Gaussian-type codes
  takes the RPA fit of VWN ("VWN-RPA": x0 = -0.409286, b = 13.0720,
  c = 42.7198); VWN's own recommended fit ("VWN5": x0 = -0.10498,
  b = 3.72744, c = 12.9352) is available as `vwn="5"`.
* LYP correlation (Lee, Yang, Parr 1988) in the form of Miehlich, Savin,
  Stoll and Preuss (1989), which integrates the Laplacian terms by parts:
    E_c = -a INT 4/(1+d rho^{-1/3}) rho_a rho_b / rho
          - a b INT w { rho_a rho_b [ 2^{11/3} C_F (rho_a^{8/3} + rho_b^{8/3})
                 + (47/18 - 7 delta/18) |grad rho|^2 - (5/2 - delta/18)(|grad rho_a|^2 + |grad rho_b|^2)
                 - ((delta - 11)/9)(rho_a/rho |grad rho_a|^2 + rho_b/rho |grad rho_b|^2) ]
               - (2/3) rho^2 |grad rho|^2 + (2/3 rho^2 - rho_a^2) |grad rho_b|^2
               + (2/3 rho^2 - rho_b^2) |grad rho_a|^2 },
    w = exp(-c rho^{-1/3}) / (1 + d rho^{-1/3}) rho^{-11/3},
    delta = c rho^{-1/3} + d rho^{-1/3} / (1 + d rho^{-1/3}),
    C_F = (3/10)(3 pi^2)^{2/3}, a = 0.04918, b = 0.132, c = 0.2533, d = 0.349.
  `lyp_original` is the 1988 closed-shell form with the Weizsaecker kinetic
  energy density and the Laplacian, used by the tests: the two forms differ
  pointwise but have the same integral.

The Kohn-Sham matrix of a GGA, V_mn = INT [ df/drho phi_m phi_n
+ 2 df/dsigma grad rho . grad(phi_m phi_n) ] (sigma = |grad rho|^2), takes
df/drho and df/dsigma from torch's automatic differentiation of the energy
densities above (CPU, float64), so the potential is the exact derivative of
the functional as written.

Grid (Becke 1988): each atom carries spherical shells of points; its share of
a point is Becke's fuzzy-cell weight (cell function s(mu) = (1 - f(f(f(mu))))/2,
f(mu) = 3mu/2 - mu^3/2, no atomic size adjustment). Radial: Becke's mapping
r = R (1 + x) / (1 - x) of Gauss-Chebyshev (second kind) nodes, R = 1 bohr
(reading). Angular: a product grid, Gauss-Legendre in cos(theta) times equally
spaced phi, exact for spherical harmonics up to degree 2 n_theta - 1 (in
place of Lebedev's grids, whose tables are not at hand).
"""
from __future__ import annotations

import math

import numpy as np

from . import rhf as R

# B3LYP mixing (Becke 1993)
A0, AX, AC = 0.20, 0.72, 0.81
B88_BETA = 0.0042
LYP_A, LYP_B, LYP_C, LYP_D = 0.04918, 0.132, 0.2533, 0.349
VWN_A = 0.0310907
VWN_PARAMS = {"rpa": (-0.409286, 13.0720, 42.7198), "5": (-0.10498, 3.72744, 12.9352)}
RHO_MIN = 1e-14   # points with less density contribute nothing


# ----------------------------------------------------------------------- grid
def radial_grid(n: int, Rm: float = 1.0):
    """Becke's radial quadrature: nodes r_i and weights w_i with
    sum_i w_i f(r_i) ~ int_0^inf f(r) r^2 dr."""
    i = np.arange(1, n + 1)
    t = i * math.pi / (n + 1)
    x = np.cos(t)
    wx = math.pi / (n + 1) * np.sin(t) ** 2 / np.sqrt(1.0 - x ** 2)   # int g(x) dx
    r = Rm * (1.0 + x) / (1.0 - x)
    drdx = 2.0 * Rm / (1.0 - x) ** 2
    return r, wx * drdx * r ** 2


def angular_grid(n_theta: int):
    """Unit vectors and weights (sum 4 pi) of the product grid."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    n_phi = 2 * n_theta
    phi = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    st = np.sqrt(1.0 - ct ** 2)
    pts = np.stack([np.outer(st, np.cos(phi)).ravel(), np.outer(st, np.sin(phi)).ravel(),
                    np.repeat(ct, n_phi)], axis=1)
    w = np.repeat(wt, n_phi) * (2.0 * math.pi / n_phi)
    return pts, w


def becke_partition(points, centres):
    """Becke's fuzzy-cell weights P_A(r) / sum_B P_B(r), [npts, natom]."""
    d = np.linalg.norm(points[:, None, :] - centres[None, :, :], axis=2)     # [npts, natom]
    nat = len(centres)
    P = np.ones((len(points), nat))
    for a in range(nat):
        for b in range(nat):
            if a == b:
                continue
            Rab = float(np.linalg.norm(centres[a] - centres[b]))
            mu = (d[:, a] - d[:, b]) / Rab
            for _ in range(3):
                mu = 1.5 * mu - 0.5 * mu ** 3
            P[:, a] *= 0.5 * (1.0 - mu)
    return P / P.sum(axis=1, keepdims=True)


def molecular_grid(xyz, n_rad: int = 75, n_theta: int = 18, Rm: float = 1.0):
    """Points [npts, 3] and weights [npts] of the molecular grid."""
    xyz = np.asarray(xyz, float)
    r, wr = radial_grid(n_rad, Rm)
    u, wu = angular_grid(n_theta)
    shell = (r[:, None, None] * u[None, :, :]).reshape(-1, 3)
    wsh = (wr[:, None] * wu[None, :]).ravel()
    pts, ws = [], []
    for a in range(len(xyz)):
        p = shell + xyz[a]
        w = wsh * becke_partition(p, xyz)[:, a]
        pts.append(p)
        ws.append(w)
    return np.concatenate(pts), np.concatenate(ws)


# ------------------------------------------------------- basis on the grid
def _cart_list(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _sph_rows(l, spherical):
    """Rows: basis functions of the shell; columns: Cartesian components
    (radial part normalised for x^l), the oracle's conventions."""
    comps = _cart_list(l)
    if spherical and l == 2:
        s3 = math.sqrt(3.0)
        return np.array([[0, s3, 0, 0, 0, 0], [0, 0, 0, 0, s3, 0], [-0.5, 0, 0, -0.5, 0, 1.0],
                         [0, 0, s3, 0, 0, 0], [0.5 * s3, 0, 0, -0.5 * s3, 0, 0]])
    if spherical and l > 2:
        raise ValueError("spherical shells above d are not supported")
    return np.diag([math.sqrt(R._dfact(2 * l - 1) / (R._dfact(2 * a - 1) * R._dfact(2 * b - 1) * R._dfact(2 * c - 1)))
                    for a, b, c in comps])


def _pow(x, n):
    return x ** n if n >= 0 else np.zeros_like(x)


_HESS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def ao_values(ob: R.OracleBasis, points, laplacian: bool = False, hessian: bool = False):
    """phi [npts, nbf], grad phi [3, npts, nbf] and (laplacian=True) the
    Laplacian [npts, nbf] of every basis function at the points; with
    hessian=True the third result is instead the second derivatives
    [6, npts, nbf] in the order xx, xy, xz, yy, yz, zz."""
    pts = np.asarray(points, float)
    npts = len(pts)
    phi = np.zeros((npts, ob.nbf))
    grad = np.zeros((3, npts, ob.nbf))
    lap = np.zeros((npts, ob.nbf)) if laplacian else None
    hes = np.zeros((6, npts, ob.nbf)) if hessian else None
    f0 = 0
    for s in range(len(ob.l)):
        l = int(ob.l[s])
        d = pts - ob.cen[s]
        r2 = np.sum(d * d, axis=1)
        p0 = int(ob.poff[s])
        a = ob.exps[p0:p0 + ob.nprim[s]]
        c = ob.coefs[p0:p0 + ob.nprim[s]]
        e = np.exp(-np.outer(r2, a))              # [npts, nprim]
        g0 = e @ c                                 # sum c e^{-a r^2}
        g1 = e @ (c * a)                           # sum c a e^{-a r^2}
        g2 = e @ (c * a * a)
        comps = _cart_list(l)
        cv = np.zeros((npts, len(comps)))
        cg = np.zeros((3, npts, len(comps)))
        cl = np.zeros((npts, len(comps)))
        ch = np.zeros((6, npts, len(comps))) if hessian else None
        for k, n in enumerate(comps):
            mono = _pow(d[:, 0], n[0]) * _pow(d[:, 1], n[1]) * _pow(d[:, 2], n[2])
            cv[:, k] = mono * g0
            for x in range(3):
                # d/dx [x^i G] = i x^{i-1} G - 2 x^{i+1} sum c a e^{-a r^2}
                lo = n[x] * _pow(d[:, x], n[x] - 1)
                rest = np.prod([_pow(d[:, y], n[y]) for y in range(3) if y != x], axis=0)
                cg[x, :, k] = rest * (lo * g0 - 2.0 * _pow(d[:, x], n[x] + 1) * g1)
            if laplacian:
                # sum_x d2/dx2 [x^i e^{-a r^2}]: (i(i-1) x^{i-2} - 2a(2i+1) x^i + 4a^2 x^{i+2}) e^{-a r^2}
                t = np.zeros(npts)
                for x in range(3):
                    rest = np.prod([_pow(d[:, y], n[y]) for y in range(3) if y != x], axis=0)
                    i = n[x]
                    t += rest * (i * (i - 1) * _pow(d[:, x], i - 2) * g0
                                 - 2.0 * (2 * i + 1) * _pow(d[:, x], i) * g1
                                 + 4.0 * _pow(d[:, x], i + 2) * g2)
                cl[:, k] = t
            if hessian:
                P = [_pow(d[:, y], n[y]) for y in range(3)]
                for hi, (x, y) in enumerate(_HESS):
                    z = 3 - x - y
                    if x == y:
                        # d2/dx2 [x^i G] = i(i-1) x^{i-2} G - 2(2i+1) x^i G1 + 4 x^{i+2} G2
                        i = n[x]
                        o = [q for q in range(3) if q != x]
                        ch[hi, :, k] = P[o[0]] * P[o[1]] * (i * (i - 1) * _pow(d[:, x], i - 2) * g0
                                                            - 2.0 * (2 * i + 1) * _pow(d[:, x], i) * g1
                                                            + 4.0 * _pow(d[:, x], i + 2) * g2)
                    else:
                        # d2/dxdy [x^i y^j G]: (i x^{i-1} - 2a x^{i+1})(j y^{j-1} - 2a y^{j+1}) per primitive
                        i, j = n[x], n[y]
                        xm, xp = i * _pow(d[:, x], i - 1), _pow(d[:, x], i + 1)
                        ym, yp = j * _pow(d[:, y], j - 1), _pow(d[:, y], j + 1)
                        ch[hi, :, k] = P[z] * (xm * ym * g0 - 2.0 * (xm * yp + xp * ym) * g1 + 4.0 * xp * yp * g2)
        T = _sph_rows(l, ob.spherical)
        nf = T.shape[0]
        phi[:, f0:f0 + nf] = cv @ T.T
        for x in range(3):
            grad[x, :, f0:f0 + nf] = cg[x] @ T.T
        if laplacian:
            lap[:, f0:f0 + nf] = cl @ T.T
        if hessian:
            for hi in range(6):
                hes[hi, :, f0:f0 + nf] = ch[hi] @ T.T
        f0 += nf
    return phi, grad, (hes if hessian else lap)


def density_on_grid(D, phi, grad, lap=None):
    """rho, grad rho [3, npts] and (lap given) the Laplacian of rho for the
    density matrix D."""
    Dphi = phi @ D
    rho = np.einsum("pm,pm->p", Dphi, phi)
    grho = 2.0 * np.einsum("pm,xpm->xp", Dphi, grad)
    lrho = None
    if lap is not None:
        lrho = 2.0 * (np.einsum("pm,pm->p", Dphi, lap) + np.sum((grad @ D) * grad, axis=(0, 2)))
    return rho, grho, lrho


# ---------------------------------------------------------------- functionals
def _torch():
    import torch
    return torch


def lda_x(rho):
    """Dirac-Slater exchange energy density (closed shell)."""
    return -0.75 * (3.0 / math.pi) ** (1.0 / 3.0) * rho ** (4.0 / 3.0)


def b88_dx(rho, sigma):
    """B88 gradient correction to exchange (closed shell), energy density."""
    torch = _torch()
    rs = rho / 2.0
    gs = torch.sqrt(sigma) / 2.0
    x = gs / rs ** (4.0 / 3.0)
    return 2.0 * (-B88_BETA * rs ** (4.0 / 3.0) * x * x / (1.0 + 6.0 * B88_BETA * x * torch.asinh(x)))


def vwn_eps(rs, kind="rpa"):
    """VWN paramagnetic correlation energy per electron at Wigner-Seitz radius rs."""
    torch = _torch()
    x0, b, c = VWN_PARAMS[kind]
    x = torch.sqrt(rs)
    X = x * x + b * x + c
    X0 = x0 * x0 + b * x0 + c
    Q = math.sqrt(4.0 * c - b * b)
    at = torch.atan(Q / (2.0 * x + b))
    return VWN_A * (torch.log(x * x / X) + 2.0 * b / Q * at
                    - b * x0 / X0 * (torch.log((x - x0) ** 2 / X) + 2.0 * (b + 2.0 * x0) / Q * at))


def vwn_c(rho, kind="rpa"):
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    return rho * vwn_eps(rs, kind)


def lyp_spin(ra, rb, gaa, gbb, gab):
    """LYP correlation energy density, Miehlich et al. form, for spin
    densities ra, rb and gradient products gaa = |grad ra|^2, gbb, gab =
    grad ra . grad rb."""
    torch = _torch()
    a, b, c, d = LYP_A, LYP_B, LYP_C, LYP_D
    rho = ra + rb
    rm = rho ** (-1.0 / 3.0)
    den = 1.0 + d * rm
    w = torch.exp(-c * rm) / den * rho ** (-11.0 / 3.0)
    delta = c * rm + d * rm / den
    CF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)
    g = gaa + gbb + 2.0 * gab
    t1 = -a * 4.0 / den * ra * rb / rho
    br = (ra * rb * (2.0 ** (11.0 / 3.0) * CF * (ra ** (8.0 / 3.0) + rb ** (8.0 / 3.0))
                     + (47.0 / 18.0 - 7.0 * delta / 18.0) * g
                     - (2.5 - delta / 18.0) * (gaa + gbb)
                     - (delta - 11.0) / 9.0 * (ra / rho * gaa + rb / rho * gbb))
          - 2.0 / 3.0 * rho * rho * g
          + (2.0 / 3.0 * rho * rho - ra * ra) * gbb
          + (2.0 / 3.0 * rho * rho - rb * rb) * gaa)
    return t1 - a * b * w * br


def lyp(rho, sigma):
    """LYP correlation energy density (closed shell, Miehlich et al. form)."""
    h = rho / 2.0
    q = sigma / 4.0
    return lyp_spin(h, h, q, q, q)


def lyp_original(rho, sigma, lap):
    """LYP 1988 closed-shell form with the Weizsaecker kinetic energy density
    t_W = |grad rho|^2 / (8 rho) - lap rho / 8 and the Laplacian:
    -a [rho + b rho^{-2/3} (C_F rho^{5/3} - 2 t_W + t_W/9 + lap rho/18) e^{-c rho^{-1/3}}] / (1 + d rho^{-1/3})."""
    torch = _torch()
    a, b, c, d = LYP_A, LYP_B, LYP_C, LYP_D
    CF = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)
    rm = rho ** (-1.0 / 3.0)
    tw = sigma / (8.0 * rho) - lap / 8.0
    inner = CF * rho ** (5.0 / 3.0) - 2.0 * tw + tw / 9.0 + lap / 18.0
    return -a * (rho + b * rho ** (-2.0 / 3.0) * inner * torch.exp(-c * rm)) / (1.0 + d * rm)


def b3lyp_density(rho, sigma, vwn="rpa"):
    """Energy density of the B3LYP exchange-correlation minus its exact-exchange part."""
    return ((1.0 - A0) * lda_x(rho) + AX * b88_dx(rho, sigma)
            + (1.0 - AC) * vwn_c(rho, vwn) + AC * lyp(rho, sigma))


# ---------------------------------------------------------- XC energy, matrix
def xc_energy_matrix(D, phi, grad, w, func=b3lyp_density):
    """E_xc = INT f(rho, sigma) and V_mn = INT [f_rho phi_m phi_n + 2 f_sigma
    grad rho . grad(phi_m phi_n)] on the grid (weights w)."""
    torch = _torch()
    rho, grho, _ = density_on_grid(D, phi, grad)
    keep = rho > RHO_MIN
    r = torch.tensor(rho[keep], dtype=torch.float64, requires_grad=True)
    s = torch.tensor(np.sum(grho[:, keep] ** 2, axis=0), dtype=torch.float64, requires_grad=True)
    f = func(r, s)
    # each point's energy density depends on that point's rho and sigma only,
    # so the gradient of the sum gives f_rho and f_sigma point by point
    fr, fs = torch.autograd.grad(f.sum(), (r, s), allow_unused=True)
    fr = fr.numpy() if fr is not None else np.zeros(len(r))
    fs = fs.numpy() if fs is not None else np.zeros(len(r))
    pk, gk, wkn = phi[keep], grad[:, keep], w[keep]
    E = float(np.sum(wkn * f.detach().numpy()))
    V = (pk * (wkn * fr)[:, None]).T @ pk
    # 2 f_sigma grad rho . (grad phi_m phi_n + phi_m grad phi_n)
    u = 2.0 * wkn * fs
    M = np.einsum("xp,xpm->pm", grho[:, keep] * u, gk)     # [p, m]
    V += M.T @ pk + pk.T @ M
    return E, V


def xc_on_grid(ob: R.OracleBasis, D, pts, w, func=b3lyp_density, chunk: int = 20000):
    """E_xc and V_xc over the grid in blocks of `chunk` points (the basis
    values of one block at a time), for molecules whose whole table of basis
    values would not fit in memory; the same sums as xc_energy_matrix."""
    E, V = 0.0, np.zeros((ob.nbf, ob.nbf))
    for a in range(0, len(w), chunk):
        phi, g, _ = ao_values(ob, pts[a:a + chunk])
        e, v = xc_energy_matrix(D, phi, g, w[a:a + chunk], func)
        E += e
        V += v
    return E, V


# ---------------------------------------------------------------------- SCF
def ks_scf(ob: R.OracleBasis, Z, xyz, grid=None, a0: float = A0, func=b3lyp_density, conv_energy=1e-10,
           conv_error=1e-8, max_iter=100, diis_size=8, tau=1e-12):
    """Closed-shell Kohn-Sham SCF with the hybrid E = sum D h + 1/2 sum D J
    - a0/4 sum D K + E_xc[rho] + V_nn, where func gives the non-exact part
    of the exchange-correlation energy density (func=None: none, so that
    a0 = 1 is RHF). DIIS on F = h + J - a0 K/2 + V_xc. Returns a dict with
    the energy, density, orbital energies, iterations and convergence."""
    nel = int(sum(int(z) for z in Z))
    if nel % 2:
        raise ValueError("closed-shell Kohn-Sham needs an even electron count")
    nocc = nel // 2
    S, T, V = R.one_electron(ob, Z, xyz)
    h = T + V
    e_nn, _ = R.nuclear_repulsion(Z, xyz)
    X = R.orthogonaliser(S)
    D = R.core_guess(h, X, nocc)
    if func is not None:
        pts, w = grid if grid is not None else molecular_grid(xyz)
        # basis values kept for the whole SCF when the table is small,
        # recomputed block by block every iteration otherwise
        whole = len(w) * ob.nbf <= 8_000_000
        if whole:
            phi, gphi, _ = ao_values(ob, pts)
    Fs, es = [], []
    E_prev = None
    converged = False
    for it in range(1, max_iter + 1):
        J, K, _ = R.jk(ob, D, tau)
        if func is None:
            Exc, Vxc = 0.0, np.zeros_like(h)
        elif whole:
            Exc, Vxc = xc_energy_matrix(D, phi, gphi, w, func)
        else:
            Exc, Vxc = xc_on_grid(ob, D, pts, w, func)
        F = h + J - 0.5 * a0 * K + Vxc
        E = float(np.sum(D * h) + 0.5 * np.sum(D * J) - 0.25 * a0 * np.sum(D * K)) + Exc + e_nn
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        emax = float(np.abs(err).max())
        if E_prev is not None and abs(E - E_prev) < conv_energy and emax < conv_error:
            converged = True
            break
        E_prev = E
        Fs.append(F)
        es.append(err)
        if len(Fs) > diis_size:
            Fs.pop(0)
            es.pop(0)
        Fbar = F
        if len(Fs) >= 2:
            m = len(Fs)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.lstsq(B, rhs, rcond=None)[0]
            Fbar = sum(c[i] * Fs[i] for i in range(m))
        eps, Cp = np.linalg.eigh(X.T @ Fbar @ X)
        C = X @ Cp
        D = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    # one last diagonalisation of F(D): orbitals, D and the energy-weighted W of the gradient
    eps, Cp = np.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    Co = C[:, :nocc]
    return dict(energy=E, D=2.0 * Co @ Co.T, W=2.0 * (Co * eps[:nocc]) @ Co.T, C=C, F=F, S=S, eps=eps,
                iterations=it, converged=converged, exc=Exc)


# ------------------------------------------------------------------ gradient
def _function_atoms(ob: R.OracleBasis):
    out = []
    for s_ in range(len(ob.l)):
        out += [int(ob.atom[s_])] * ob.shell_nbf(s_)
    return np.array(out)


def xc_gradient(ob: R.OracleBasis, natom, D, pts, w, func=b3lyp_density, chunk: int = 20000):
    """d E_xc / dA on a grid fixed in space (the weights do not move with the
    atoms): rho and grad rho change only through the basis functions of A,
    d phi_m / dA = -grad phi_m for m on A, so
      d rho / dA_x = -2 sum_{m on A} d_x phi_m (D phi)_m,
      d (d_y rho) / dA_x = -2 sum_{m on A} [d_x d_y phi_m (D phi)_m + d_x phi_m (D d_y phi)_m],
    and dE_xc/dA_x = INT [f_rho d rho/dA_x + 2 f_sigma grad rho . d grad rho / dA_x]."""
    torch = _torch()
    fat = _function_atoms(ob)
    g = np.zeros((natom, 3))
    for a in range(0, len(w), chunk):
        phi, gp, hs = ao_values(ob, pts[a:a + chunk], hessian=True)
        wk = w[a:a + chunk]
        rho, grho, _ = density_on_grid(D, phi, gp)
        keep = rho > RHO_MIN
        phi, gp, hs, wk, rho, grho = phi[keep], gp[:, keep], hs[:, keep], wk[keep], rho[keep], grho[:, keep]
        r = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
        s_ = torch.tensor(np.sum(grho ** 2, axis=0), dtype=torch.float64, requires_grad=True)
        fr, fs = torch.autograd.grad(func(r, s_).sum(), (r, s_), allow_unused=True)
        fr = fr.numpy() if fr is not None else np.zeros(len(wk))
        fs = fs.numpy() if fs is not None else np.zeros(len(wk))
        Dphi = phi @ D                       # (D phi)_m at each point
        Dg = gp @ D                          # (D d_y phi)_m, [3, p, m]
        per_m = np.zeros((3, ob.nbf))
        for x in range(3):
            drho = -2.0 * gp[x] * Dphi       # per-function pieces of d rho / dA_x
            acc = (wk * fr) @ drho
            for y in range(3):
                hi = _HESS.index((min(x, y), max(x, y)))
                dgy = -2.0 * (hs[hi] * Dphi + gp[x] * Dg[y])
                acc += (wk * 2.0 * fs * grho[y]) @ dgy
            per_m[x] = acc
        for x in range(3):
            np.add.at(g[:, x], fat, per_m[x])
    return g


def b3lyp_energy_gradient(basis: dict, Z, xyz, grid=None, tau: float = 1e-12, **kw):
    """B3LYP energy (Eh) and gradient dE/dR (Eh/bohr) on a grid fixed in space
    (default: the molecular grid at these coordinates): one-electron terms
    with the Kohn-Sham W, the two-electron gradient with 20% exact exchange,
    the XC gradient (xc_gradient) and dV_nn/dR."""
    ob = R.OracleBasis.build(basis, Z, xyz)
    pts, w = grid if grid is not None else molecular_grid(xyz)
    res = ks_scf(ob, Z, xyz, grid=(pts, w), tau=tau, **kw)
    D, W = res["D"], res["W"]
    g = (R.grad_1e(ob, Z, xyz, D, W) + R.grad_2e(ob, len(Z), D, tau, kx=A0)
         + xc_gradient(ob, len(Z), D, pts, w) + R.nuclear_repulsion(Z, xyz)[1])
    return res["energy"], g, res
