"""The allocation-free eigensolver entry point (pimd_eigh_noalloc) against the
context-based one (pimd_eigh_dev), called through the C ABI.

pimd_eigh_noalloc exists for callers that cannot allocate device memory (their
GPU memory belongs to another allocator, or their loop must not take the
device synchronisation of cudaMalloc/cudaFree); it keeps its workspace in a
fixed device array. This file is collected last so that a failure here stops
a first-failure run only after every other test has run.
"""
import numpy as np
import pytest

from paper_1601_02713_gb300 import native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _matrices(nmat, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(nmat, n, n))
    A = A + A.transpose(0, 2, 1)
    A[:, range(n), range(n)] += np.linspace(-30, 60, n)  # Fock-like spread of the spectrum
    return A


def _both(ctx, A):
    """Eigenpairs of the batch A from both entry points (noalloc on a side
    stream, read after that stream has finished)."""
    nmat, n = A.shape[0], A.shape[1]
    At = torch.tensor(A, device="cuda")
    V0, w0 = torch.empty_like(At), torch.empty(nmat, n, dtype=torch.float64, device="cuda")
    V1, w1 = torch.empty_like(At), torch.empty(nmat, n, dtype=torch.float64, device="cuda")
    native.pimd_eigh_dev(ctx, At, V0, w0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    rc = native.pimd_eigh_noalloc(At, V1, w1, stream=s.cuda_stream)
    s.synchronize()
    assert rc == native.PIMD_OK
    return (w0.cpu().numpy(), V0.cpu().numpy()), (w1.cpu().numpy(), V1.cpu().numpy())


def _compare(A, r0, r1):
    (w0, V0), (w1, V1) = r0, r1
    nmat, n = A.shape[0], A.shape[1]
    scale = np.abs(A).max()
    np.testing.assert_allclose(w1, w0, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(w1, np.linalg.eigvalsh(A), rtol=0, atol=1e-10 * scale)
    for k in range(nmat):
        # same eigenvectors up to sign: compare the reconstructions
        R0 = (V0[k] * w0[k]) @ V0[k].T
        R1 = (V1[k] * w1[k]) @ V1[k].T
        np.testing.assert_allclose(R1, R0, rtol=0, atol=1e-10 * scale)
        np.testing.assert_allclose(V1[k].T @ V1[k], np.eye(n), rtol=0, atol=1e-12)


def test_noalloc_eigensolver_matches_context_solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = native.Context(0)
    for nmat, n, seed in [(3, 40, 1), (5, 33, 2)]:  # two calls in a row, odd and even n
        A = _matrices(nmat, n, seed)
        r0, r1 = _both(ctx, A)
        _compare(A, r0, r1)


def test_noalloc_at_its_limits():
    """Batches at the workspace's limits: 1024 matrices (the descriptor
    limit) of n = 45 (2,073,600 doubles, just under 2,097,152)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = native.Context(0)
    A = _matrices(1024, 45, 7)
    r0, r1 = _both(ctx, A)
    _compare(A[:16], (r0[0][:16], r0[1][:16]), (r1[0][:16], r1[1][:16]))
    np.testing.assert_allclose(r1[0], r0[0], rtol=0, atol=1e-11 * np.abs(A).max())


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for nmat, n in [(3, 1000), (4, 768), (1025, 2)]:   # n limit; doubles limit at n = 768; descriptor limit
        A = torch.zeros(nmat, n, n, dtype=torch.float64, device="cuda")
        V = torch.empty_like(A)
        w = torch.empty(nmat, n, dtype=torch.float64, device="cuda")
        assert native.pimd_eigh_noalloc(A, V, w) == native.PIMD_EINVAL
