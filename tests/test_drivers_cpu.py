"""Replica drivers around the force step (CPU, with model potentials in
place of the GPU forces call): ring-polymer PIMD (normal modes, exact free
ring-polymer propagation, NVE energy conservation with second-order error,
PILE-L thermostat equipartition) and the string method (equal-arc-length
reparametrisation; convergence to a minimum-energy path on the Mueller-Brown
surface, whose gradient is then parallel to the path)."""
import math

import numpy as np
import pytest

from paper_1601_02713_gb300 import drivers as DR


def morse_forces(De=0.17, a=1.2, re=1.8):
    """E and dE/dq of every bead for a Morse bond between atoms 0 and 1 of
    each bead (q [P, N, 3], bohr)."""
    def fn(q):
        d = q[:, 0] - q[:, 1]
        r = np.linalg.norm(d, axis=1)
        e = np.exp(-a * (r - re))
        E = De * (1 - e) ** 2
        dEdr = 2 * De * a * e * (1 - e)
        G = np.zeros_like(q)
        G[:, 0] = (dEdr / r)[:, None] * d
        G[:, 1] = -G[:, 0]
        return E, G
    return fn


def _ring(P=8, T=300.0, dt=0.5 * DR.FS, thermostat=False, seed=1, tau0=100.0 * DR.FS):
    rng = np.random.default_rng(seed)
    q = np.array([[0.0, 0.0, 0.0], [1.8, 0.0, 0.0]])[None] + 0.05 * rng.normal(size=(P, 2, 3))
    return DR.RingPolymer([8, 1], q, T, dt, thermostat=thermostat, seed=seed, tau0=tau0)


@pytest.mark.parametrize("P", [1, 2, 5, 8])
def test_normal_modes_diagonalise_the_ring(P):
    C = DR.normal_mode_matrix(P)
    np.testing.assert_allclose(C.T @ C, np.eye(P), atol=1e-13)
    wP = 0.7
    A = wP ** 2 * (2 * np.eye(P) - np.roll(np.eye(P), 1, axis=0) - np.roll(np.eye(P), -1, axis=0))
    if P == 1:
        A = np.zeros((1, 1))
    M = C.T @ A @ C
    np.testing.assert_allclose(M, np.diag(DR.mode_frequencies(P, wP) ** 2), atol=1e-12)


def test_free_ring_polymer_is_propagated_exactly():
    """With V = 0 the A step is exact: kinetic + spring energy is conserved
    to round-off at any time step, and the centroid moves uniformly."""
    rp = _ring(P=6, dt=5.0 * DR.FS)
    zero = lambda q: (np.zeros(len(q)), np.zeros_like(q))
    rp.evaluate(zero)
    H0 = rp.hamiltonian()
    c0 = rp.q.mean(0)
    v = (rp.p.sum(0) / rp.P) / rp.m[:, None]
    for _ in range(50):
        rp.step(zero)
    assert abs(rp.hamiltonian() - H0) < 1e-12 * abs(H0)
    np.testing.assert_allclose(rp.q.mean(0), c0 + 50 * rp.dt * v, atol=1e-9)


def test_nve_conserves_the_ring_polymer_energy_to_second_order():
    drift = []
    for dt in (0.5 * DR.FS, 0.25 * DR.FS):
        rp = _ring(dt=dt)
        fn = morse_forces()
        rp.evaluate(fn)
        H0 = rp.hamiltonian()
        dev = 0.0
        for _ in range(int(round(40 * DR.FS / dt))):
            rp.step(fn)
            dev = max(dev, abs(rp.hamiltonian() - H0))
        drift.append(dev)
    assert drift[0] < 1e-3                      # hartree over 40 fs at 0.5 fs (H ~ 0.25)
    assert 3.0 < drift[0] / drift[1] < 5.5      # error of second order in dt


def test_thermostat_equipartition_of_the_ring():
    """PILE-L samples the ring-polymer momenta at the temperature P T: the
    mean kinetic energy per degree of freedom is 1 / (2 beta_P)."""
    rp = _ring(P=4, T=300.0, dt=0.5 * DR.FS, thermostat=True, seed=3, tau0=5.0 * DR.FS)
    fn = morse_forces()
    ke = []
    for i in range(6000):
        rp.step(fn)
        if i >= 500:
            ke.append(rp.kinetic())
    ndof = rp.P * rp.N * 3
    assert np.mean(ke) / (ndof / (2 * rp.beta_P)) == pytest.approx(1.0, abs=0.03)


def test_reparametrisation_equalises_arc_length():
    rng = np.random.default_rng(0)
    t = np.sort(rng.uniform(0, 1, 12))
    t[0], t[-1] = 0.0, 1.0
    curve = np.stack([np.cos(2 * t), np.sin(2 * t), t], axis=1)   # images unevenly spaced on a helix arc
    out = DR.reparametrize(curve)
    s = DR.arc_lengths(out)
    seg = np.diff(s)
    # equal spacing along the piecewise-linear string through the input images
    s_in = DR.arc_lengths(curve)
    assert abs(s[-1] - s_in[-1]) < 1e-2 * s_in[-1]   # chords of the polyline: slightly shorter
    assert seg.max() - seg.min() < 0.05 * seg.mean()
    np.testing.assert_allclose(out[0], curve[0])
    np.testing.assert_allclose(out[-1], curve[-1])
    line = np.linspace(0, 1, 7)[:, None] * np.array([[1.0, 2.0, -1.0]]) ** 1
    line2 = line[[0, 1, 3, 4, 6]]
    np.testing.assert_allclose(DR.reparametrize(line2), np.linspace(0, 1, 5)[:, None] * np.array([[1.0, 2.0, -1.0]]),
                               atol=1e-14)


MB_A = (-200.0, -100.0, -170.0, 15.0)
MB_a = (-1.0, -1.0, -6.5, 0.7)
MB_b = (0.0, 0.0, 11.0, 0.6)
MB_c = (-10.0, -10.0, -6.5, 0.7)
MB_x0 = (1.0, 0.0, -0.5, -1.0)
MB_y0 = (0.0, 0.5, 1.5, 1.0)


def mueller_brown(x):
    """The Mueller-Brown model surface (Theor. Chim. Acta 53, 75 (1979)) and
    its gradient, for images x [n, 2]."""
    x = np.asarray(x, float).reshape(-1, 2)
    E = np.zeros(len(x))
    G = np.zeros_like(x)
    for A, a, b, c, x0, y0 in zip(MB_A, MB_a, MB_b, MB_c, MB_x0, MB_y0):
        dx, dy = x[:, 0] - x0, x[:, 1] - y0
        e = A * np.exp(a * dx * dx + b * dx * dy + c * dy * dy)
        E += e
        G[:, 0] += e * (2 * a * dx + b * dy)
        G[:, 1] += e * (b * dx + 2 * c * dy)
    return E, G


def test_mueller_brown_gradient_is_its_derivative():
    x = np.array([[0.1, 0.4], [-0.6, 1.2], [0.5, 0.1]])
    E, G = mueller_brown(x)
    h = 1e-6
    for k in range(2):
        d = np.zeros(2)
        d[k] = h
        fd = (mueller_brown(x + d)[0] - mueller_brown(x - d)[0]) / (2 * h)
        np.testing.assert_allclose(G[:, k], fd, rtol=1e-6, atol=1e-6)


def test_string_converges_to_a_minimum_energy_path():
    """From a straight line between two points near the deep minima, the
    string relaxes (ends included) into the path through the intermediate
    minimum; at convergence the gradient at every image is parallel to the
    path, and the highest image sits where the gradient nearly vanishes."""
    a, b = np.array([-0.55, 1.45]), np.array([0.62, 0.03])
    n = 24
    x0 = a + np.linspace(0, 1, n)[:, None] * (b - a)
    sm = DR.StringMethod(x0, dt=2e-4)
    E0, G0 = mueller_brown(x0)
    gperp0 = sm.perpendicular_gradient(G0)
    for _ in range(6000):
        sm.step(mueller_brown)
    E, G = mueller_brown(sm.x)
    gperp = sm.perpendicular_gradient(G)
    scale = np.abs(G0).max()
    # with 24 images the tangent's discretisation leaves a perpendicular part
    # of at most ~20% of |grad| where the path bends; the straight start had 100%
    assert gperp.max() < 0.15 * gperp0.max()
    assert np.all(gperp[1:-1] < 0.25 * np.linalg.norm(G[1:-1], axis=1))
    seg = np.diff(DR.arc_lengths(sm.x))
    assert seg.max() - seg.min() < 0.05 * seg.mean()   # equal arc length up to the chords cutting corners
    # ends relaxed into minima
    assert np.abs(G[0]).max() < 1e-3 * scale and np.abs(G[-1]).max() < 1e-3 * scale
    # a barrier along the path, well below the straight line's highest point
    k = int(np.argmax(E[1:-1])) + 1
    assert E[k] > max(E[0], E[-1]) and E[k] < E0.max()
    assert np.linalg.norm(G[k]) < 0.1 * scale
