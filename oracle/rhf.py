"""Oracle RHF driver (numpy) over the McMurchie-Davidson integrals of
integrals.c. TEST INFRASTRUCTURE ONLY (see the package docstring).

Steps, in the textbook order of the closed-shell Roothaan-Hall method:

1. contracted Gaussians normalised (primitive norm, then contraction norm);
2. S, T, V; h = T + V; nuclear repulsion V_nn;
3. orthogonaliser X = S^{-1/2} (canonical, dropping eigenvalues < 1e-8, if S
   is nearly singular);
4. core-Hamiltonian guess;
5. loop: F = h + J - K/2; E = 1/2 sum D (h + F) + V_nn;
   e = X^T (F D S - S D F) X; stop when |dE| < conv_energy and max|e| <
   conv_error; Pulay DIIS on (F, e) (subspace 8); F' = X^T F X; eigh; aufbau;
   D = 2 C_occ C_occ^T;
6. gradient with D and W = 2 C_occ diag(eps_occ) C_occ^T from one last
   diagonalisation of F(D):
   g_A = sum D dh/dA - sum W dS/dA + 1/2 sum (D D - D D / 2) d(mn|ls)/dA
         + dV_nn/dA.

The paper's thresholds (Sec. 3.1): integral cutoff 1e-12 on the Schwarz
bound; its SCF density threshold 1e-6 is tightened to |dE| < 1e-10 and
max|e| < 1e-8 so that energies and forces are converged well inside the
parity tolerances (1e-8 Eh, 1e-6 Eh/bohr).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "integrals.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile integrals.c with gcc (OpenMP, -O2, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        basis = [ctypes.c_int, ip, ip, ip, dp, dp, dp, ip, ctypes.c_int]
        lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double]
        lib.oracle_boys.restype = ctypes.c_double
        lib.oracle_eri_block.argtypes = basis + [ctypes.c_int] * 4 + [dp]
        lib.oracle_schwarz.argtypes = basis + [dp]
        lib.oracle_eri_full.argtypes = basis + [dp]
        lib.oracle_jk.argtypes = basis + [dp, ctypes.c_double, dp, dp]
        lib.oracle_jk.restype = ctypes.c_longlong
        lib.oracle_grad_2e.argtypes = basis + [ctypes.c_int, dp, ctypes.c_double, dp]
        lib.oracle_grad_2e_kx.argtypes = basis + [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_one_electron.argtypes = basis + [ctypes.c_int, dp, dp, dp, dp, dp]
        lib.oracle_grad_1e.argtypes = basis + [ctypes.c_int, dp, dp, dp, dp, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_g_block.argtypes = basis + [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_eri_list.argtypes = basis + [ctypes.c_int, ip]
        lib.oracle_eri_list.restype = ctypes.c_double
        lib.oracle_deriv_list.argtypes = basis + [ctypes.c_int, ip]
        lib.oracle_deriv_list.restype = ctypes.c_double
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return _load().oracle_num_threads()


def boys(m: int, T: float) -> float:
    """F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt."""
    return _load().oracle_boys(int(m), float(T))


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def normalise_shell(l: int, exps, coefs) -> np.ndarray:
    """Contraction coefficients that normalise the axis-aligned component x^l
    of the contracted shell: primitive norm
      N(a, l) = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!)
    then the contraction rescaled so that <phi|phi> = 1, using
      <g_a|g_b> (x^l component) = (pi/(a+b))^{3/2} (2l-1)!! / (2(a+b))^l."""
    a = np.asarray(exps, float)
    c = np.asarray(coefs, float) * (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(_dfact(2 * l - 1))
    s = a[:, None] + a[None, :]
    ov = (math.pi / s) ** 1.5 * _dfact(2 * l - 1) / (2 * s) ** l
    return c / math.sqrt(float(c @ ov @ c))


@dataclass
class OracleBasis:
    """Shells of one molecule (per-atom expansion of a per-element basis)."""
    l: np.ndarray
    nprim: np.ndarray
    poff: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray
    cen: np.ndarray
    atom: np.ndarray
    spherical: int
    nbf: int

    @classmethod
    def build(cls, basis: dict, Z, xyz, spherical: bool = True) -> "OracleBasis":
        ls, nps, po, ex, co, ce, at = [], [], [], [], [], [], []
        p = 0
        nbf = 0
        for ia, z in enumerate(Z):
            for sh in basis[int(z)]:
                ls.append(sh.l)
                nps.append(len(sh.exps))
                po.append(p)
                p += len(sh.exps)
                ex.extend(sh.exps)
                co.extend(normalise_shell(sh.l, sh.exps, sh.coefs))
                ce.append(np.asarray(xyz[ia], float))
                at.append(ia)
                nbf += (2 * sh.l + 1) if (spherical and sh.l >= 2) else (sh.l + 1) * (sh.l + 2) // 2
        return cls(np.array(ls, np.int32), np.array(nps, np.int32), np.array(po, np.int32),
                   np.array(ex, float), np.array(co, float), np.ascontiguousarray(np.array(ce, float)),
                   np.array(at, np.int32), int(bool(spherical)), nbf)

    def args(self):
        return (len(self.l), _ip(self.l), _ip(self.nprim), _ip(self.poff), _dp(self.exps),
                _dp(self.coefs), _dp(self.cen), _ip(self.atom), self.spherical)

    def shell_nbf(self, s):
        l = int(self.l[s])
        return 2 * l + 1 if (self.spherical and l >= 2) else (l + 1) * (l + 2) // 2


def eri_block(ob: OracleBasis, a, b, c, d) -> np.ndarray:
    n = [ob.shell_nbf(s) for s in (a, b, c, d)]
    out = np.zeros(n)
    _load().oracle_eri_block(*ob.args(), a, b, c, d, _dp(out))
    return out


def eri_full(ob: OracleBasis) -> np.ndarray:
    N = ob.nbf
    out = np.zeros((N, N, N, N))
    _load().oracle_eri_full(*ob.args(), _dp(out))
    return out


def schwarz(ob: OracleBasis) -> np.ndarray:
    ns = len(ob.l)
    Q = np.zeros((ns, ns))
    _load().oracle_schwarz(*ob.args(), _dp(Q))
    return Q


def one_electron(ob: OracleBasis, Z, xyz):
    N = ob.nbf
    S, T, V = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
    Zn = np.asarray(Z, float)
    C = np.ascontiguousarray(np.asarray(xyz, float))
    _load().oracle_one_electron(*ob.args(), len(Zn), _dp(Zn), _dp(C), _dp(S), _dp(T), _dp(V))
    return S, T, V


def jk(ob: OracleBasis, D, tau: float = 1e-12):
    """J_mn = sum D_ls (mn|ls), K_mn = sum D_ls (ml|ns); Schwarz cutoff tau
    on Q_ab Q_cd (Sec. 3.1: integral cutoff 1e-12). Returns (J, K, nquartets)."""
    N = ob.nbf
    D = np.ascontiguousarray(D, float)
    J, K = np.zeros((N, N)), np.zeros((N, N))
    nq = _load().oracle_jk(*ob.args(), _dp(D), float(tau), _dp(J), _dp(K))
    return J, K, nq


def grad_2e(ob: OracleBasis, natom, D, tau: float = 1e-12, kx: float = 1.0):
    """Two-electron gradient 1/2 sum (D_mn D_ls - kx/2 D_ml D_ns) d(mn|ls)/dA
    (kx = 1: Hartree-Fock; a hybrid's fraction of exact exchange otherwise)."""
    g = np.zeros((natom, 3))
    D = np.ascontiguousarray(D, float)
    if kx == 1.0:
        _load().oracle_grad_2e(*ob.args(), natom, _dp(D), float(tau), _dp(g))
    else:
        _load().oracle_grad_2e_kx(*ob.args(), natom, _dp(D), float(tau), float(kx), _dp(g))
    return g


def grad_1e(ob: OracleBasis, Z, xyz, D, W):
    natom = len(Z)
    g = np.zeros((natom, 3))
    Zn = np.asarray(Z, float)
    C = np.ascontiguousarray(np.asarray(xyz, float))
    _load().oracle_grad_1e(*ob.args(), natom, _dp(Zn), _dp(C), _dp(np.ascontiguousarray(D, float)),
                           _dp(np.ascontiguousarray(W, float)), _dp(g))
    return g


def g_block(ob: OracleBasis, D, a: int, b: int) -> np.ndarray:
    """Block of G = J - K/2 for shells a, b from the definitions, summed over
    every ordered shell pair without screening (sampled checks of large
    systems)."""
    out = np.zeros((ob.shell_nbf(a), ob.shell_nbf(b)))
    _load().oracle_g_block(*ob.args(), _dp(np.ascontiguousarray(D, float)), int(a), int(b), _dp(out))
    return out


def eri_list(ob: OracleBasis, quartets) -> float:
    """Contracted blocks of the listed shell quartets (timing samples)."""
    q = np.ascontiguousarray(quartets, np.int32)
    return _load().oracle_eri_list(*ob.args(), len(q), _ip(q))


def deriv_list(ob: OracleBasis, quartets) -> float:
    """Derivative blocks of the listed shell quartets (timing samples)."""
    q = np.ascontiguousarray(quartets, np.int32)
    return _load().oracle_deriv_list(*ob.args(), len(q), _ip(q))


def canonical_quartets(ob: OracleBasis, tau: float = 1e-12):
    """All canonical shell quartets (a>=b, c>=d, ab>=cd) with Q_ab Q_cd >= tau,
    as an [n, 4] int array (pair order as in oracle_jk)."""
    Q = schwarz(ob)
    ns = len(ob.l)
    a, b = np.tril_indices(ns)
    qp = Q[a, b]
    out = []
    for i in range(len(a)):
        j = np.nonzero(qp[: i + 1] * qp[i] >= tau)[0]
        if len(j):
            out.append(np.stack([np.full(len(j), a[i]), np.full(len(j), b[i]), a[j], b[j]], axis=1))
    return np.concatenate(out).astype(np.int32)


def nuclear_repulsion(Z, xyz):
    """V_nn = sum_{A<B} Z_A Z_B / R_AB and its gradient."""
    Z = np.asarray(Z, float)
    R = np.asarray(xyz, float)
    E = 0.0
    g = np.zeros_like(R)
    for A in range(len(Z)):
        for B in range(A):
            d = R[A] - R[B]
            r = math.sqrt(float(d @ d))
            E += Z[A] * Z[B] / r
            g[A] -= Z[A] * Z[B] * d / r ** 3
            g[B] += Z[A] * Z[B] * d / r ** 3
    return E, g


def orthogonaliser(S, drop: float = 1e-8):
    """Symmetric (Loewdin) S^{-1/2}; canonical S-eigenvector orthogonalisation
    with eigenvalues below `drop` removed when S is nearly singular."""
    s, U = np.linalg.eigh(S)
    if s.min() >= drop:
        return (U / np.sqrt(s)) @ U.T
    keep = s >= drop
    return U[:, keep] / np.sqrt(s[keep])


def core_guess(h, X, nocc):
    e, Cp = np.linalg.eigh(X.T @ h @ X)
    C = X @ Cp
    return 2.0 * C[:, :nocc] @ C[:, :nocc].T


@dataclass
class SCFResult:
    energy: float
    D: np.ndarray
    W: np.ndarray
    C: np.ndarray
    eps: np.ndarray
    iterations: int
    converged: bool
    S: np.ndarray
    h: np.ndarray
    F: np.ndarray
    e_nn: float
    nquartets: int
    homo_lumo_gap: float


def run_scf(ob: OracleBasis, Z, xyz, conv_energy=1e-10, conv_error=1e-8, max_iter=100,
            diis_size=8, tau=1e-12, D0=None, verbose=False) -> SCFResult:
    nel = int(sum(int(z) for z in Z))
    if nel % 2:
        raise ValueError("closed-shell RHF needs an even electron count")
    nocc = nel // 2
    S, T, V = one_electron(ob, Z, xyz)
    h = T + V
    e_nn, _ = nuclear_repulsion(Z, xyz)
    X = orthogonaliser(S)
    D = core_guess(h, X, nocc) if D0 is None else np.array(D0, float)
    Fs, es = [], []
    E_prev = None
    converged = False
    nq = 0
    for it in range(1, max_iter + 1):
        J, K, nq = jk(ob, D, tau)
        F = h + J - 0.5 * K
        E = 0.5 * float(np.sum(D * (h + F))) + e_nn
        err = X.T @ (F @ D @ S - S @ D @ F) @ X
        emax = float(np.abs(err).max())
        if verbose:
            print(f"it {it:3d} E {E:.12f} dE {E - (E_prev or 0):.3e} |e| {emax:.3e}")
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
        while len(Fs) >= 2:
            m = len(Fs)
            B = -np.ones((m + 1, m + 1))
            B[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(B, rhs)
            except np.linalg.LinAlgError:
                Fs.pop(0)
                es.pop(0)
                continue
            Fbar = sum(c[i] * Fs[i] for i in range(m))
            break
        eps, Cp = np.linalg.eigh(X.T @ Fbar @ X)
        C = X @ Cp
        D = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    # one last diagonalisation of F(D) for the orbitals, D and W of the gradient
    eps, Cp = np.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    Co = C[:, :nocc]
    Dg = 2.0 * Co @ Co.T
    W = 2.0 * (Co * eps[:nocc]) @ Co.T
    gap = float(eps[nocc] - eps[nocc - 1]) if len(eps) > nocc else float("nan")
    return SCFResult(E, Dg, W, C, eps, it, converged, S, h, F, e_nn, nq, gap)


def sad_atomic_density(basis: dict, Z: int, tol: float = 1e-9, max_iter: int = 200) -> np.ndarray:
    """Spherically averaged density of the isolated neutral atom Z (<= 10) in
    `basis`, the building block of the superposition-of-atomic-densities
    guess (the paper has no such guess; it reuses the previous step's MOs).

    Configuration 1s^2 2s^2 2p^(Z-4): the first two s orbitals (lowest orbital
    energies among the s-type eigenvectors) take min(electrons left, 2) each,
    the electrons left after them are shared evenly by the three lowest p-type
    eigenvectors. Orbitals are told apart by angular momentum, not energy
    order (in a fractional-occupation SCF the 2s can lie above the 2p).
    Iterate F = h + J(D) - K(D)/2 -> eigenvectors -> D = sum_k n_k C_k C_k^T,
    starting from the eigenvectors of h, until max|D_new - D| < tol.
    """
    Zs = np.array([Z], np.int32)
    xyz = np.zeros((1, 3))
    ob = OracleBasis.build(basis, Zs, xyz)
    S, T, V = one_electron(ob, Zs, xyz)
    h = T + V
    X = orthogonaliser(S)
    lfun = np.concatenate([[sh.l] * (2 * sh.l + 1) for sh in basis[int(Z)]])

    def occupied_density(F):
        eps, Cp = np.linalg.eigh(X.T @ F @ X)
        C = X @ Cp
        lk = [int(np.argmax([np.sum(C[lfun == l, k] ** 2) for l in range(3)])) for k in range(C.shape[1])]
        n = np.zeros(C.shape[1])
        left = int(Z)
        s_orb = [k for k in np.argsort(eps, kind="stable") if lk[k] == 0][:2]
        p_orb = [k for k in np.argsort(eps, kind="stable") if lk[k] == 1][:3]
        for k in s_orb:
            n[k] = min(left, 2)
            left -= int(n[k])
        if left > 0:
            if len(p_orb) < 3 or left > 6:
                raise ValueError("configuration needs a 2p shell")
            n[p_orb] = left / 3.0
        return (C * n) @ C.T

    D = occupied_density(h)
    for _ in range(max_iter):
        J, K, _ = jk(ob, D)
        Dn = occupied_density(h + J - 0.5 * K)
        diff = float(np.abs(Dn - D).max())
        D = Dn
        if diff < tol:
            break
    return D


def rhf_energy_gradient(basis: dict, Z, xyz, want_gradient=True, tau=1e-12, **kw):
    """Converged RHF energy (Eh) and gradient dE/dR (Eh/bohr, [natom, 3])."""
    ob = OracleBasis.build(basis, Z, xyz)
    res = run_scf(ob, Z, xyz, tau=tau, **kw)
    if not want_gradient:
        return res.energy, None, res
    g = grad_1e(ob, Z, xyz, res.D, res.W) + grad_2e(ob, len(Z), res.D, tau) + nuclear_repulsion(Z, xyz)[1]
    return res.energy, g, res
