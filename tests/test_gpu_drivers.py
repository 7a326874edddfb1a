"""Replica drivers with the GPU force step (through the C ABI): a
ring-polymer PIMD trajectory of the water dimer (4 beads, minimal basis)
conserves the ring-polymer energy with a second-order error in the time
step, and string-method steps on water-dimer images lower the images'
energies while keeping them equally spaced."""
import numpy as np
import pytest

from paper_1601_02713_gb300 import drivers as DR
from paper_1601_02713_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reps, kind = inputs.workload("water2_min_4beads")
    Z, X = reps.stacked()
    ctx = native.Context(0)
    B = native.Basis(inputs.basis_set(kind))
    return ctx, B, Z, X


def test_pimd_nve_with_bo_forces(setup):
    """NVE ring-polymer dynamics on the BO surface: the drift of the
    ring-polymer energy over 2 fs falls by four when the time step halves
    (the splitting is of second order; the beads start 0.1 A from each other,
    so the motion is large and the error is measured at small steps)."""
    ctx, B, Z, X = setup
    fn = DR.bo_forces_fn(ctx, B, Z)
    drift = []
    for dt in (0.2 * DR.FS, 0.1 * DR.FS, 0.05 * DR.FS):
        ctx.clear_guess()
        rp = DR.RingPolymer(Z, X, 300.0, dt, thermostat=False, seed=7)
        rp.evaluate(fn)
        H0 = rp.hamiltonian()
        dev = 0.0
        for _ in range(int(round(2 * DR.FS / dt))):
            rp.step(fn)
            dev = max(dev, abs(rp.hamiltonian() - H0))
        drift.append(dev)
    assert 3.0 < drift[0] / drift[1] < 5.5, drift
    assert 3.0 < drift[1] / drift[2] < 5.5, drift


def test_string_steps_with_bo_forces(setup):
    ctx, B, Z, X = setup
    # four images between two beads of the dimer (same atoms, different geometry)
    images = X[0][None] + np.linspace(0.0, 1.0, 4)[:, None, None] * (X[3] - X[0])[None]
    fn = DR.images_forces_fn(ctx, B, Z)
    sm = DR.StringMethod(images, dt=0.2)
    E0 = sm.step(fn)
    for _ in range(4):
        E = sm.step(fn)
    assert E.sum() < E0.sum()
    seg = np.diff(DR.arc_lengths(sm.x))
    assert seg.max() - seg.min() < 0.05 * seg.mean()
