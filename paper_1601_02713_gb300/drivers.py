"""Replica dynamics around the force step: path-integral molecular dynamics
of a ring polymer (the paper's PIMD, Sec. 2) and the string method for a
reaction path (Sec. 3.2). Both are host-side drivers: each step calls one
forces function for all replicas at once (on the GPU, `pimd_bo_forces` or
`string_images_forces` of the C ABI, see `bo_forces_fn`) and then moves the
replicas, so the step time is the forces call plus a few array operations.

Units: atomic units throughout (bohr, hartree, electron masses, hbar = 1,
time in hbar/hartree); `AMU`, `FS` and `KB` convert.
"""
from __future__ import annotations

import math

import numpy as np

AMU = 1822.888486209         # electron masses per unified atomic mass unit
FS = 41.341373335            # atomic time units per femtosecond
KB = 3.166811563e-6          # Boltzmann constant, hartree per kelvin
MASS_AMU = {1: 1.00782503223, 6: 12.0, 8: 15.99491461957}   # most abundant isotopes


def masses_au(Z) -> np.ndarray:
    return np.array([MASS_AMU[int(z)] * AMU for z in Z])


# --------------------------------------------------------------------------
# Ring-polymer PIMD
# --------------------------------------------------------------------------
def normal_mode_matrix(P: int) -> np.ndarray:
    """Orthogonal C [P, P] (bead k, mode j) that diagonalises the ring's
    nearest-neighbour spring matrix: mode 0 is the centroid 1/sqrt(P);
    1 <= j < P/2 sqrt(2/P) cos(2 pi j k / P); j = P/2 (P even) (-1)^k/sqrt(P);
    P/2 < j < P sqrt(2/P) sin(2 pi j k / P). Mode j has the free ring-polymer
    frequency 2 omega_P sin(pi j / P)."""
    k = np.arange(P)
    C = np.zeros((P, P))
    for j in range(P):
        if j == 0:
            C[:, j] = 1.0 / math.sqrt(P)
        elif 2 * j < P:
            C[:, j] = math.sqrt(2.0 / P) * np.cos(2 * math.pi * j * k / P)
        elif 2 * j == P:
            C[:, j] = (-1.0) ** k / math.sqrt(P)
        else:
            C[:, j] = math.sqrt(2.0 / P) * np.sin(2 * math.pi * j * k / P)
    return C


def mode_frequencies(P: int, omega_P: float) -> np.ndarray:
    return 2.0 * omega_P * np.sin(math.pi * np.arange(P) / P)


class RingPolymer:
    """P beads of an N-atom molecule at temperature T (kelvin): positions q
    and momenta p [P, N, 3]. The ring-polymer Hamiltonian is
      H = sum_k sum_i p_ki^2 / (2 m_i) + 1/2 m_i omega_P^2 |q_ki - q_k+1,i|^2
          + sum_k V(q_k),   omega_P = P k_B T / hbar,
    integrated by the symmetric splitting O(dt/2) B(dt/2) A(dt) B(dt/2) O(dt/2):
    B a half kick by the physical forces of every bead, A the exact evolution
    of the free ring polymer in its normal modes, O the path-integral Langevin
    thermostat (PILE-L: friction 2 omega_j on mode j > 0 and 1/tau0 on the
    centroid; Ceriotti, Parrinello, Markland, Manolopoulos, J. Chem. Phys. 133,
    124104 (2010)) at the ring temperature P T. thermostat=False gives NVE
    dynamics, which conserves H."""

    def __init__(self, Z, q, T: float, dt: float, thermostat: bool = True, tau0: float = 100.0 * FS,
                 seed: int = 0):
        self.Z = np.asarray(Z)
        self.q = np.array(q, dtype=np.float64)
        self.P, self.N = self.q.shape[0], self.q.shape[1]
        self.m = masses_au(self.Z)
        self.beta_P = 1.0 / (KB * T * self.P)
        self.omega_P = 1.0 / self.beta_P
        self.dt = float(dt)
        self.C = normal_mode_matrix(self.P)
        self.w = mode_frequencies(self.P, self.omega_P)
        self.thermostat = thermostat
        gam = np.where(np.arange(self.P) == 0, 1.0 / tau0, 2.0 * self.w)
        self.c1 = np.exp(-0.5 * self.dt * gam)
        self.c2 = np.sqrt(1.0 - self.c1 ** 2)
        self.rng = np.random.default_rng(seed)
        self.p = self.sample_momenta()
        self.E = None
        self.G = None

    # normal-mode transforms over the bead axis
    def to_modes(self, x):
        return np.einsum("kj,kia->jia", self.C, x)

    def to_beads(self, x):
        return np.einsum("kj,jia->kia", self.C, x)

    def sample_momenta(self):
        return self.rng.normal(size=self.q.shape) * np.sqrt(self.m / self.beta_P)[None, :, None]

    def kinetic(self):
        return float(np.sum(self.p ** 2 / (2.0 * self.m[None, :, None])))

    def spring(self):
        d = self.q - np.roll(self.q, -1, axis=0)
        return float(0.5 * self.omega_P ** 2 * np.sum(self.m[None, :, None] * d ** 2))

    def hamiltonian(self):
        """Ring-polymer H (conserved without the thermostat); needs the
        energies of the current positions (after `step` or `evaluate`)."""
        return self.kinetic() + self.spring() + float(np.sum(self.E))

    def evaluate(self, forces_fn):
        self.E, self.G = forces_fn(self.q)
        self.E = np.asarray(self.E, dtype=np.float64)
        self.G = np.asarray(self.G, dtype=np.float64).reshape(self.q.shape)

    def _O(self):
        if not self.thermostat:
            return
        pm = self.to_modes(self.p)
        xi = self.rng.normal(size=pm.shape)
        pm = self.c1[:, None, None] * pm + self.c2[:, None, None] * np.sqrt(self.m / self.beta_P)[None, :, None] * xi
        self.p = self.to_beads(pm)

    def _A(self):
        qm, pm = self.to_modes(self.q), self.to_modes(self.p)
        m = self.m[None, :, None]
        for j in range(self.P):
            if self.w[j] == 0.0:
                qm[j] = qm[j] + pm[j] * self.dt / m[0]
                continue
            c, s = math.cos(self.w[j] * self.dt), math.sin(self.w[j] * self.dt)
            mw = m[0] * self.w[j]
            pj = c * pm[j] - mw * s * qm[j]
            qj = s / mw * pm[j] + c * qm[j]
            pm[j], qm[j] = pj, qj
        self.q, self.p = self.to_beads(qm), self.to_beads(pm)

    def step(self, forces_fn):
        """One time step; forces_fn(q [P, N, 3]) -> (E [P], dE/dq [P, N, 3])."""
        if self.G is None:
            self.evaluate(forces_fn)
        self._O()
        self.p -= 0.5 * self.dt * self.G
        self._A()
        self.evaluate(forces_fn)
        self.p -= 0.5 * self.dt * self.G
        self._O()

    def centroid_virial_kinetic(self):
        """Centroid-virial estimator of the quantum kinetic energy:
        3 N / (2 beta) + 1/(2P) sum_k (q_k - q_c) . dV/dq_k."""
        qc = self.q.mean(axis=0, keepdims=True)
        beta = self.beta_P * self.P
        return 1.5 * self.N / beta + 0.5 / self.P * float(np.sum((self.q - qc) * self.G))


# --------------------------------------------------------------------------
# String method
# --------------------------------------------------------------------------
def arc_lengths(images) -> np.ndarray:
    """Cumulative arc length s_i of the piecewise-linear string through the
    images [n, ...] (s_0 = 0)."""
    x = np.asarray(images, dtype=np.float64).reshape(len(images), -1)
    seg = np.sqrt(np.sum(np.diff(x, axis=0) ** 2, axis=1))
    return np.concatenate([[0.0], np.cumsum(seg)])


def reparametrize(images) -> np.ndarray:
    """Images redistributed at equal arc length along the piecewise-linear
    string through the given ones (end points kept)."""
    x = np.asarray(images, dtype=np.float64)
    shape = x.shape
    x = x.reshape(len(x), -1)
    s = arc_lengths(x)
    if s[-1] == 0.0:
        return x.reshape(shape).copy()
    t = np.linspace(0.0, s[-1], len(x))
    out = np.empty_like(x)
    for d in range(x.shape[1]):
        out[:, d] = np.interp(t, s, x[:, d])
    out[0], out[-1] = x[0], x[-1]
    return out.reshape(shape)


class StringMethod:
    """The simplified string method (E, Ren, Vanden-Eijnden, J. Chem. Phys.
    126, 164103 (2007)): every image moves down its own gradient for a
    pseudo-time dt (the end images too, unless fixed_ends), then the images
    are redistributed at equal arc length. At convergence the string is a
    minimum-energy path: the gradient at each image is parallel to the path.
    The images' forces come from one call for all images (the paper evaluates
    them in parallel, Sec. 3.2)."""

    def __init__(self, images, dt: float, fixed_ends: bool = False):
        self.x = np.array(images, dtype=np.float64)
        self.dt = float(dt)
        self.fixed_ends = fixed_ends
        self.E = None
        self.G = None

    def step(self, forces_fn):
        """forces_fn(images [n, ...]) -> (E [n], dE/dx [n, ...])."""
        E, G = forces_fn(self.x)
        self.E = np.asarray(E, dtype=np.float64)
        self.G = np.asarray(G, dtype=np.float64).reshape(self.x.shape)
        move = self.dt * self.G
        if self.fixed_ends:
            move[0] = 0.0
            move[-1] = 0.0
        self.x = reparametrize(self.x - move)
        return self.E

    def tangents(self):
        x = self.x.reshape(len(self.x), -1)
        t = np.zeros_like(x)
        t[1:-1] = x[2:] - x[:-2]
        t[0] = x[1] - x[0]
        t[-1] = x[-1] - x[-2]
        return t / np.linalg.norm(t, axis=1, keepdims=True)

    def perpendicular_gradient(self, G=None):
        """|component of dE/dx perpendicular to the string| per image."""
        g = (self.G if G is None else np.asarray(G)).reshape(len(self.x), -1)
        t = self.tangents()
        gp = g - np.sum(g * t, axis=1, keepdims=True) * t
        return np.linalg.norm(gp, axis=1)


# --------------------------------------------------------------------------
# the GPU force step as a forces function
# --------------------------------------------------------------------------
def bo_forces_fn(ctx, basis, Z, opts=None):
    """forces_fn for RingPolymer: every bead of one molecule in one
    pimd_bo_forces call (guess: the previous step's MOs of each bead)."""
    from . import native
    o = opts or native.scf_opts(guess=1)

    def fn(q):
        E, G, info, rc = native.pimd_bo_forces(ctx, basis, Z, q, o)
        if rc != 0:
            raise native.PimdError(rc, "pimd_bo_forces")
        return E, G
    return fn


def images_forces_fn(ctx, basis, Z, opts=None):
    """forces_fn for StringMethod: every image (same molecule) in one
    string_images_forces call."""
    from . import native
    o = opts or native.scf_opts(guess=1)
    Z = np.asarray(Z, np.int32)

    def fn(x):
        n = len(x)
        nat = np.full(n, len(Z), np.int32)
        E, G, info, rc = native.string_images_forces(ctx, basis, nat, np.tile(Z, n), np.asarray(x).reshape(-1, 3), o)
        if rc != 0:
            raise native.PimdError(rc, "string_images_forces")
        return E, G.reshape(n, len(Z), 3)
    return fn
