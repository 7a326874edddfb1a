"""Force-parallel split of every replica (the paper's force groups): two
processes' worth of the work, run here as two host threads with one context
each on the same GPU. Each evaluates every second quartet tile, and the
partial Fock matrices (every SCF iteration) and two-electron gradients are
summed between them on the host (no kernel waits on another). The energies
and gradients must equal an unsplit call's, and both halves must take the
same SCF path."""
import threading

import numpy as np
import pytest

from paper_1601_02713_gb300 import inputs, native
from paper_1601_02713_gb300 import replicas as RP

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_two_way_split_equals_unsplit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reps, kind = inputs.workload("water8_spd_32beads", nrep=2)
    Z, X = reps.stacked()
    B = native.Basis(inputs.basis_set(kind))
    c0 = native.Context(0)
    E0, G0, i0, rc = native.pimd_bo_forces(c0, B, Z, X, native.scf_opts(guess=4))   # also uploads the tapes
    assert rc == 0
    ts = RP.ThreadSum(2)
    ctxs = [native.Context(0), native.Context(0)]
    out = [None, None]

    def run(r):
        o = native.scf_opts(guess=4, split_size=2, split_rank=r, reduce=ts.fn(r))
        out[r] = native.pimd_bo_forces(ctxs[r], B, Z, X, o, check=False)

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    for r in range(2):
        E, G, info, rc = out[r]
        assert rc == 0, native.load().pimd_last_error(ctxs[r].handle)
        assert [i["iterations"] for i in info] == [i["iterations"] for i in out[0][2]]
        np.testing.assert_allclose(E, E0, atol=1e-9, rtol=0)
        np.testing.assert_allclose(G, G0, atol=1e-8, rtol=0)
    # the same reduced Fock matrices on both: energies agree to the last bits of
    # the nuclear repulsion (summed with FP64 atomics in each context)
    np.testing.assert_allclose(out[0][0], out[1][0], atol=1e-12, rtol=0)
