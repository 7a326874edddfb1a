"""Thin ctypes binding of the C ABI in include/pimdgb.h (argument marshalling
only: every step of the computation runs in the CUDA library).

The library must have been built (`paper_1601_02713_gb300.build.build()` or
`__graft_entry__.build()`); loading fails loudly otherwise. There is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

PIMD_OK, PIMD_EINVAL, PIMD_ENOMEM, PIMD_ECUDA, PIMD_ENOTCONV, PIMD_ETIMEOUT, PIMD_EBASIS = 0, -1, -2, -3, -4, -5, -6


# reduce_fn of the force-parallel split: int fn(double* buf, long long n, void* user)
REDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p)


class PimdScfOpts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("conv_energy", ctypes.c_double),
                ("conv_error", ctypes.c_double), ("max_iter", ctypes.c_int), ("diis_size", ctypes.c_int),
                ("schwarz_tau", ctypes.c_double), ("fp32_tau", ctypes.c_double), ("guess", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("want_gradient", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("full_every", ctypes.c_int), ("prim_screen", ctypes.c_double), ("reuse_mode", ctypes.c_int),
                ("split_size", ctypes.c_int), ("split_rank", ctypes.c_int), ("reduce_fn", REDUCE_FN),
                ("reduce_user", ctypes.c_void_p)]


class PimdInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("final_dE", ctypes.c_double),
                ("final_error", ctypes.c_double), ("nquartets", ctypes.c_longlong),
                ("nq_fp64", ctypes.c_longlong), ("nq_fp32", ctypes.c_longlong)]


class PimdStats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_longlong), ("fock_builds", ctypes.c_int),
                ("ms_fock", ctypes.c_double), ("ms_grad2e", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("nquartets_total", ctypes.c_longlong), ("eri_flops_per_build", ctypes.c_double),
                ("eris_per_build", ctypes.c_double), ("eri_flops32_per_build", ctypes.c_double),
                ("quartets_fp64", ctypes.c_longlong), ("quartets_fp32", ctypes.c_longlong),
                ("eris32_per_build", ctypes.c_double), ("grad_flops", ctypes.c_double),
                ("grad_flops32", ctypes.c_double), ("grad_quartets", ctypes.c_longlong)]


class PimdError(RuntimeError):
    def __init__(self, code, what="", detail=""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" + (f" [{detail}]" if detail else ""))


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    lib.pimd_scf_opts_default.argtypes = [ctypes.POINTER(PimdScfOpts)]
    lib.pimd_scf_opts_default.restype = None
    lib.pimd_ctx_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int]
    lib.pimd_ctx_destroy.argtypes = [_P]
    lib.pimd_ctx_destroy.restype = None
    lib.pimd_ctx_clear_guess.argtypes = [_P]
    lib.pimd_ctx_clear_guess.restype = None
    lib.pimd_basis_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, _I, _I, _I, _I, _D, _D, ctypes.c_int]
    lib.pimd_basis_destroy.argtypes = [_P]
    lib.pimd_basis_destroy.restype = None
    lib.pimd_basis_nbf.argtypes = [_P, ctypes.c_int, _I]
    lib.pimd_bo_forces.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I, _D, _P, ctypes.POINTER(PimdScfOpts), _D, _D,
                                   ctypes.POINTER(PimdInfo)]
    lib.string_images_forces.argtypes = [_P, ctypes.c_int, _I, _I, _D, _P, ctypes.POINTER(PimdScfOpts), _D, _D,
                                         ctypes.POINTER(PimdInfo)]
    lib.pimd_bo_forces_dev.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I, _P, _P, ctypes.POINTER(PimdScfOpts),
                                       _P, _P, ctypes.POINTER(PimdInfo), _P]
    lib.string_images_forces_dev.argtypes = [_P, ctypes.c_int, _I, _I, _P, _P, ctypes.POINTER(PimdScfOpts), _P, _P,
                                             ctypes.POINTER(PimdInfo), _P]
    lib.pimd_last_stats.argtypes = [_P, ctypes.POINTER(PimdStats)]
    lib.pimd_screened_quartets.argtypes = [_P, ctypes.c_int, _I, _I, _D, _P, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_longlong)]
    lib.pimd_last_trace.argtypes = [_P, ctypes.c_int, ctypes.c_int, _D, _D, _I]
    lib.pimd_last_fock_times.argtypes = [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_longlong)]
    lib.pimd_fock_dev.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I, _D, _P, ctypes.c_double, ctypes.c_double, _P, _P]
    lib.pimd_one_electron.argtypes = [_P, ctypes.c_int, _I, _D, _P, _D, _D, _D]
    lib.pimd_boys_dev.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P]
    lib.pimd_boys_f32_dev.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int]
    lib.pimd_peak_bench.argtypes = [ctypes.c_int, _D, _D, _D]
    lib.pimd_eigh_dev.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
    lib.pimd_eigh_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]
    _F = ctypes.POINTER(ctypes.c_float)
    _LL = ctypes.POINTER(ctypes.c_longlong)
    lib.pimd_guess_create.argtypes = [ctypes.POINTER(_P), _P, ctypes.c_ulonglong]
    lib.pimd_guess_destroy.argtypes = [_P]
    lib.pimd_guess_destroy.restype = None
    lib.pimd_guess_nparam.argtypes = [_P]
    lib.pimd_guess_nparam.restype = ctypes.c_longlong
    lib.pimd_guess_ndata.argtypes = [_P]
    lib.pimd_guess_ndata.restype = ctypes.c_longlong
    lib.pimd_guess_clear_data.argtypes = [_P]
    lib.pimd_guess_clear_data.restype = None
    lib.pimd_guess_add_data.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _I, _D, _P, ctypes.POINTER(PimdScfOpts),
                                        _P]
    lib.pimd_guess_train.argtypes = [_P, ctypes.c_int, ctypes.c_double, _D]
    lib.pimd_guess_loss.argtypes = [_P, _D]
    lib.pimd_guess_save.argtypes = [_P, ctypes.c_char_p]
    lib.pimd_guess_load.argtypes = [_P, ctypes.c_char_p]
    lib.pimd_ctx_set_guess_model.argtypes = [_P, _P]
    lib.pimd_guess_pair_data.argtypes = [_P, ctypes.c_int, _I, _D, _D, _F, ctypes.c_int, ctypes.c_longlong, _I, _I,
                                         _LL, _F, _D, _F, _D]
    lib.pimd_guess_mlp_grad.argtypes = [_P, ctypes.c_int, ctypes.c_int, _F, _F, _D, _F, _F]
    lib.pimd_sad_atomic_density.argtypes = [_P, _P, ctypes.c_int, _D, ctypes.c_int]
    lib.pimd_autotune.argtypes = [_P, ctypes.c_int, ctypes.c_int, _I, _D, _P, ctypes.POINTER(PimdScfOpts), _I, _D]
    lib.pimd_bf16_gemm_dev.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P,
                                       ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P]
    lib.pimd_strerror.argtypes = [ctypes.c_int]
    lib.pimd_strerror.restype = ctypes.c_char_p
    lib.pimd_last_error.argtypes = [_P]
    lib.pimd_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().pimd_strerror(int(code)).decode()


def _dp(a):
    return a.ctypes.data_as(_D)


def _ip(a):
    return a.ctypes.data_as(_I)


def _check(rc, what, allow_notconv=False, ctx=None):
    if rc == PIMD_OK or (allow_notconv and rc == PIMD_ENOTCONV):
        return rc
    detail = ""
    if ctx is not None and getattr(ctx, "handle", None):
        detail = load().pimd_last_error(ctx.handle).decode()
    raise PimdError(rc, what, detail)


def scf_opts(**kw) -> PimdScfOpts:
    """Defaults of pimd_scf_opts_default, overridden by keyword. For the
    force-parallel split pass reduce=<python function (ptr, n) -> None> (it
    is wrapped as reduce_fn and kept alive with the options)."""
    o = PimdScfOpts()
    load().pimd_scf_opts_default(ctypes.byref(o))
    reduce = kw.pop("reduce", None)
    for k, v in kw.items():
        setattr(o, k, v)
    if reduce is not None:
        def _cb(ptr, n, user):
            try:
                reduce(int(ptr), int(n))
                return 0
            except Exception:   # an error must reach the library as a status, not unwind through C
                return 1
        o._reduce_cb = REDUCE_FN(_cb)
        o.reduce_fn = o._reduce_cb
    return o


class Context:
    """pimd_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.handle = _P()
        _check(load().pimd_ctx_create(ctypes.byref(self.handle), int(device)), "pimd_ctx_create")

    def close(self):
        if self.handle:
            load().pimd_ctx_destroy(self.handle)
            self.handle = _P()

    def clear_guess(self):
        load().pimd_ctx_clear_guess(self.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Basis:
    """pimd_basis from a per-element basis ({Z: [Shell(l, exps, coefs)]})."""

    def __init__(self, basis: dict):
        from .inputs import basis_arrays
        Zs, nsh, sl, snp, ex, co = basis_arrays(basis)
        self.handle = _P()
        _check(load().pimd_basis_create(ctypes.byref(self.handle), len(Zs), _ip(Zs), _ip(nsh), _ip(sl), _ip(snp),
                                        _dp(ex), _dp(co), 1), "pimd_basis_create")

    def nbf(self, Z) -> int:
        Z = np.ascontiguousarray(Z, np.int32)
        n = load().pimd_basis_nbf(self.handle, len(Z), _ip(Z))
        if n < 0:
            raise PimdError(n, "pimd_basis_nbf")
        return n

    def __del__(self):
        try:
            if self.handle:
                load().pimd_basis_destroy(self.handle)
        except Exception:
            pass


def _infos(arr):
    return [dict(iterations=i.iterations, converged=i.converged, final_dE=i.final_dE, final_error=i.final_error,
                 nquartets=i.nquartets, nq_fp64=i.nq_fp64, nq_fp32=i.nq_fp32) for i in arr]


def pimd_bo_forces(ctx: Context, basis: Basis, Z, coords, opts: PimdScfOpts | None = None, check=True):
    """Energies [nrep] and gradients [nrep, natom, 3] of nrep replicas of one
    molecule (host arrays in and out). Returns (E, G, info, rc)."""
    Z = np.ascontiguousarray(Z, np.int32)
    X = np.ascontiguousarray(coords, np.float64)
    nrep, natom = X.shape[0], X.shape[1]
    opts = opts or scf_opts()
    E = np.zeros(nrep)
    G = np.zeros((nrep, natom, 3))
    info = (PimdInfo * nrep)()
    rc = load().pimd_bo_forces(ctx.handle, nrep, natom, _ip(Z), _dp(X), basis.handle, ctypes.byref(opts), _dp(E),
                               _dp(G), info)
    if check:
        _check(rc, "pimd_bo_forces", allow_notconv=True, ctx=ctx)
    return E, G, _infos(info), rc


def string_images_forces(ctx: Context, basis: Basis, natom_of_img, Z_concat, coords_concat,
                         opts: PimdScfOpts | None = None, check=True):
    nat = np.ascontiguousarray(natom_of_img, np.int32)
    Z = np.ascontiguousarray(Z_concat, np.int32)
    X = np.ascontiguousarray(coords_concat, np.float64)
    nimg = len(nat)
    opts = opts or scf_opts()
    E = np.zeros(nimg)
    G = np.zeros((int(nat.sum()), 3))
    info = (PimdInfo * nimg)()
    rc = load().string_images_forces(ctx.handle, nimg, _ip(nat), _ip(Z), _dp(X), basis.handle, ctypes.byref(opts),
                                     _dp(E), _dp(G), info)
    if check:
        _check(rc, "string_images_forces", allow_notconv=True, ctx=ctx)
    return E, G, _infos(info), rc


def pimd_bo_forces_dev(ctx: Context, basis: Basis, Z, coords_dev, energies_dev, gradients_dev,
                       opts: PimdScfOpts | None = None, stream: int = 0, check=True):
    """Device variant: coords/energies/gradients are CUDA tensors (float64,
    contiguous) or raw device addresses."""
    Z = np.ascontiguousarray(Z, np.int32)
    nrep, natom = int(coords_dev.shape[0]), int(coords_dev.shape[1])
    opts = opts or scf_opts()
    info = (PimdInfo * nrep)()
    rc = load().pimd_bo_forces_dev(ctx.handle, nrep, natom, _ip(Z), _P(coords_dev.data_ptr()), basis.handle,
                                   ctypes.byref(opts), _P(energies_dev.data_ptr()),
                                   _P(gradients_dev.data_ptr() if gradients_dev is not None else 0), info,
                                   _P(stream))
    if check:
        _check(rc, "pimd_bo_forces_dev", allow_notconv=True, ctx=ctx)
    return _infos(info), rc


def string_images_forces_dev(ctx: Context, basis: Basis, natom_of_img, Z_concat, coords_dev, energies_dev,
                             gradients_dev, opts: PimdScfOpts | None = None, stream: int = 0, check=True):
    nat = np.ascontiguousarray(natom_of_img, np.int32)
    Z = np.ascontiguousarray(Z_concat, np.int32)
    opts = opts or scf_opts()
    info = (PimdInfo * len(nat))()
    rc = load().string_images_forces_dev(ctx.handle, len(nat), _ip(nat), _ip(Z), _P(coords_dev.data_ptr()),
                                         basis.handle, ctypes.byref(opts), _P(energies_dev.data_ptr()),
                                         _P(gradients_dev.data_ptr() if gradients_dev is not None else 0), info,
                                         _P(stream))
    if check:
        _check(rc, "string_images_forces_dev", allow_notconv=True, ctx=ctx)
    return _infos(info), rc


def pimd_fock_dev(ctx: Context, basis: Basis, Z, coords, D_dev, G_dev, schwarz_tau: float = 1e-12,
                  fp32_tau: float = 0.0):
    """G = J - K/2 of a given density for nrep replicas (D, G device tensors
    [nrep, N, N]); coords host [nrep, natom, 3]."""
    Z = np.ascontiguousarray(Z, np.int32)
    X = np.ascontiguousarray(coords, np.float64)
    _check(load().pimd_fock_dev(ctx.handle, X.shape[0], X.shape[1], _ip(Z), _dp(X), basis.handle,
                                float(schwarz_tau), float(fp32_tau), _P(D_dev.data_ptr()), _P(G_dev.data_ptr())),
           "pimd_fock_dev")


def pimd_one_electron(ctx: Context, basis: Basis, Z, coords):
    Z = np.ascontiguousarray(Z, np.int32)
    X = np.ascontiguousarray(coords, np.float64)
    N = basis.nbf(Z)
    S, T, V = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
    _check(load().pimd_one_electron(ctx.handle, len(Z), _ip(Z), _dp(X), basis.handle, _dp(S), _dp(T), _dp(V)),
           "pimd_one_electron")
    return S, T, V


def pimd_boys_dev(ctx: Context, T_dev, m: int, F_dev):
    _check(load().pimd_boys_dev(ctx.handle, int(T_dev.numel()), int(m), _P(T_dev.data_ptr()),
                                _P(F_dev.data_ptr())), "pimd_boys_dev")


def pimd_boys_f32_dev(ctx: Context, T_dev, m: int, F_dev, variant: int = 0):
    """FP32 Boys evaluation of the mixed-precision quartets (float32 CUDA
    tensors; variant 0 straight-line form, 1 cooperative-kernel form)."""
    _check(load().pimd_boys_f32_dev(ctx.handle, int(T_dev.numel()), int(m), _P(T_dev.data_ptr()),
                                    _P(F_dev.data_ptr()), int(variant)), "pimd_boys_f32_dev")


def pimd_sad_atomic_density(ctx: Context, basis: Basis, Z: int):
    """Atomic density of element Z used by the SAD guess ([n, n] host array)."""
    n = basis.nbf([Z])
    D = np.zeros((n, n))
    _check(load().pimd_sad_atomic_density(ctx.handle, basis.handle, int(Z), _dp(D), n), "pimd_sad_atomic_density")
    return D


def pimd_autotune(ctx: Context, basis: Basis, Z, coords, opts: PimdScfOpts | None = None):
    """Pick the Fock-build kernel (tile width 32/64/128, or 0 = cooperative)
    and the gradient kernel (0 cooperative, 1 straight-line) per class pair
    for this workload; returns (fock [21], grad [21], ms of one build)."""
    Z = np.ascontiguousarray(Z, np.int32)
    X = np.ascontiguousarray(coords, np.float64)
    opts = opts or scf_opts()
    w = np.zeros(64, np.int32)
    ms = np.zeros(1)
    _check(load().pimd_autotune(ctx.handle, X.shape[0], X.shape[1], _ip(Z), _dp(X), basis.handle,
                                ctypes.byref(opts), _ip(w), _dp(ms)), "pimd_autotune")
    return w[:21].tolist(), w[32:53].tolist(), float(ms[0])


def pimd_bf16_gemm_dev(A, B, C, ta: bool, tb: bool, stream: int = 0) -> int:
    """C = op(A) op(B) for bf16 CUDA tensors A, B (row-major) into the float32
    CUDA tensor C [M, N] on the tensor cores; returns the status code."""
    M, N = int(C.shape[0]), int(C.shape[1])
    K = int(A.shape[0] if ta else A.shape[1])
    return load().pimd_bf16_gemm_dev(M, N, K, _P(A.data_ptr()), int(A.stride(0)), int(ta), _P(B.data_ptr()),
                                     int(B.stride(0)), int(tb), _P(C.data_ptr()), int(C.stride(0)), _P(stream))


def pimd_screened_quartets(ctx: Context, basis: Basis, natom_of_img, Z_concat, coords_concat,
                           schwarz_tau: float = 1e-12) -> np.ndarray:
    """Screened shell quartets per replica (host arrays, layout of
    string_images_forces)."""
    nat = np.ascontiguousarray(natom_of_img, np.int32)
    Z = np.ascontiguousarray(Z_concat, np.int32)
    X = np.ascontiguousarray(coords_concat, np.float64)
    out = np.zeros(len(nat), np.int64)
    _check(load().pimd_screened_quartets(ctx.handle, len(nat), _ip(nat), _ip(Z), _dp(X), basis.handle,
                                         float(schwarz_tau), out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))),
           "pimd_screened_quartets")
    return out


def pimd_last_trace(ctx: Context, rep: int) -> dict:
    """Per-iteration energy, error and full-build flag of replica rep in the
    last forces call."""
    lib = load()
    n = lib.pimd_last_trace(ctx.handle, int(rep), 0, None, None, None)
    if n < 0:
        raise PimdError(n, "pimd_last_trace")
    E, err, full = np.zeros(max(n, 1)), np.zeros(max(n, 1)), np.zeros(max(n, 1), np.int32)
    lib.pimd_last_trace(ctx.handle, int(rep), n, _dp(E), _dp(err), _ip(full))
    return {"energy": E[:n], "error": err[:n], "full_build": full[:n]}


def pimd_last_fock_times(ctx: Context) -> dict:
    """Per SCF iteration of the last forces call: device time (ms) of the
    Fock build and the shell quartets it executed."""
    lib = load()
    n = lib.pimd_last_fock_times(ctx.handle, 0, None, None)
    if n < 0:
        raise PimdError(n, "pimd_last_fock_times")
    ms, q = np.zeros(max(n, 1)), np.zeros(max(n, 1), np.int64)
    lib.pimd_last_fock_times(ctx.handle, n, _dp(ms), q.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return {"ms": ms[:n], "quartets": q[:n]}


def pimd_last_stats(ctx: Context) -> dict:
    s = PimdStats()
    _check(load().pimd_last_stats(ctx.handle, ctypes.byref(s)), "pimd_last_stats")
    return {k: getattr(s, k) for k, _ in PimdStats._fields_}


def eigh_args_ok(A_dev, V_dev, evals_dev) -> bool:
    """True if A [nmat, n, n], V [nmat, n, n] and evals [nmat, n] are
    contiguous float64 CUDA tensors on one device (checked before any launch:
    the eigensolver reads and writes exactly these extents)."""
    try:
        import torch
    except ImportError:
        return False
    ts = (A_dev, V_dev, evals_dev)
    if not all(isinstance(t, torch.Tensor) for t in ts):
        return False
    if A_dev.dim() != 3 or A_dev.shape[1] != A_dev.shape[2]:
        return False
    nmat, n = int(A_dev.shape[0]), int(A_dev.shape[1])
    if nmat <= 0 or n <= 0:
        return False
    if tuple(V_dev.shape) != (nmat, n, n) or tuple(evals_dev.shape) != (nmat, n):
        return False
    if any(t.dtype != torch.float64 or not t.is_contiguous() for t in ts):
        return False
    return all(t.is_cuda for t in ts) and len({t.device for t in ts}) == 1


def pimd_eigh_dev(ctx: Context, A_dev, V_dev, evals_dev, stream: int = 0):
    """Batched symmetric eigensolver (context workspace). A, V: [nmat, n, n]
    and evals: [nmat, n], contiguous float64 CUDA tensors (PimdError with
    PIMD_EINVAL otherwise, before anything is launched)."""
    if not eigh_args_ok(A_dev, V_dev, evals_dev):
        raise PimdError(PIMD_EINVAL, "pimd_eigh_dev: A, V [nmat,n,n] and evals [nmat,n] must be contiguous "
                                     "float64 CUDA tensors on one device")
    nmat, n = int(A_dev.shape[0]), int(A_dev.shape[1])
    _check(load().pimd_eigh_dev(ctx.handle, nmat, n, _P(A_dev.data_ptr()), _P(V_dev.data_ptr()),
                                _P(evals_dev.data_ptr()), _P(stream)), "pimd_eigh_dev")


def pimd_eigh_noalloc(A_dev, V_dev, evals_dev, stream: int = 0):
    """The same eigensolver without any device allocation (fixed 16 MiB
    device workspace; nmat * n * n <= 2,097,152, nmat <= 1024); it only
    enqueues its kernels on `stream`. Returns the status code (PIMD_EINVAL,
    without a launch, unless A, V [nmat, n, n] and evals [nmat, n] are
    contiguous float64 CUDA tensors on one device)."""
    if not eigh_args_ok(A_dev, V_dev, evals_dev):
        return PIMD_EINVAL
    nmat, n = int(A_dev.shape[0]), int(A_dev.shape[1])
    return load().pimd_eigh_noalloc(nmat, n, _P(A_dev.data_ptr()), _P(V_dev.data_ptr()), _P(evals_dev.data_ptr()),
                                    _P(stream))


def pimd_peak_bench(device: int = 0) -> dict:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().pimd_peak_bench(int(device), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "pimd_peak_bench")
    return {"fp64_tflops": a.value, "fp32_tflops": b.value, "dmma_fp64_tflops": c.value}


_FP = ctypes.POINTER(ctypes.c_float)


def _fp(a):
    return a.ctypes.data_as(_FP) if a is not None else None


class GuessModel:
    """pimd_guess: the learned initial density (model, training set and
    training on the device of the current CUDA device)."""

    NTYPE = 9
    NF = 96

    def __init__(self, basis: Basis, seed: int = 0):
        self.handle = _P()
        _check(load().pimd_guess_create(ctypes.byref(self.handle), basis.handle, int(seed)), "pimd_guess_create")

    @property
    def nparam(self) -> int:
        return int(load().pimd_guess_nparam(self.handle))

    @property
    def ndata(self) -> int:
        return int(load().pimd_guess_ndata(self.handle))

    def add_data(self, ctx: Context, basis: Basis, Z, coords, opts: PimdScfOpts | None = None):
        """Converge the SCF of the replicas coords[nrep, natom, 3] and add their
        densities to the training set; returns the per-replica info."""
        Z = np.ascontiguousarray(Z, np.int32)
        X = np.ascontiguousarray(coords, np.float64)
        opts = opts or scf_opts()
        info = (PimdInfo * X.shape[0])()
        _check(load().pimd_guess_add_data(self.handle, ctx.handle, X.shape[0], X.shape[1], _ip(Z), _dp(X),
                                          basis.handle, ctypes.byref(opts), ctypes.cast(info, _P)),
               "pimd_guess_add_data", ctx=ctx)
        return _infos(info)

    def clear_data(self):
        load().pimd_guess_clear_data(self.handle)

    def train(self, epochs: int, lr: float = 1e-3) -> np.ndarray:
        hist = np.zeros(max(int(epochs), 1))
        _check(load().pimd_guess_train(self.handle, int(epochs), float(lr), _dp(hist)), "pimd_guess_train")
        return hist[:int(epochs)]

    def loss(self) -> float:
        v = np.zeros(1)
        _check(load().pimd_guess_loss(self.handle, _dp(v)), "pimd_guess_loss")
        return float(v[0])

    def save(self, path: str):
        _check(load().pimd_guess_save(self.handle, str(path).encode()), "pimd_guess_save")

    def load_weights(self, path: str):
        _check(load().pimd_guess_load(self.handle, str(path).encode()), "pimd_guess_load")

    def attach(self, ctx: Context):
        """Use this model for guess = 2 and 3 in ctx (the model must outlive
        its use there)."""
        _check(load().pimd_ctx_set_guess_model(ctx.handle, self.handle), "pimd_ctx_set_guess_model")

    def pair_data(self, Z, coords, D=None, local_in=None, nbf=None):
        """Test hook: pair rows of one molecule. Returns dict with pairs [n,2],
        block_off [n], feats [n,96], frames [n,3,3], local (if D) and D_lab
        (if local_in)."""
        Z = np.ascontiguousarray(Z, np.int32)
        X = np.ascontiguousarray(coords, np.float64)
        n_at = len(Z)
        npmax = n_at * (n_at + 1) // 2
        noutmax = npmax * 14 * 14
        npair = ctypes.c_int()
        AB = np.zeros((npmax, 2), np.int32)
        off = np.zeros(npmax, np.int64)
        feats = np.zeros((npmax, self.NF), np.float32)
        frames = np.zeros((npmax, 9))
        Dh = np.ascontiguousarray(D, np.float64) if D is not None else None
        loc_out = np.zeros(noutmax, np.float32) if D is not None else None
        loc_in = None
        Dout = None
        if local_in is not None:
            loc_in = np.zeros(noutmax, np.float32)
            loc_in[:len(local_in)] = local_in
            N = int(nbf) if nbf is not None else int(Dh.shape[0])
            Dout = np.zeros((N, N))
        rc = load().pimd_guess_pair_data(self.handle, n_at, _ip(Z), _dp(X), _dp(Dh) if Dh is not None else None,
                                         _fp(loc_in), npmax, noutmax, ctypes.byref(npair), _ip(AB),
                                         off.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), _fp(feats),
                                         _dp(frames), _fp(loc_out), _dp(Dout) if Dout is not None else None)
        _check(rc, "pimd_guess_pair_data")
        n = npair.value
        out = dict(pairs=AB[:n].copy(), block_off=off[:n].copy(), feats=feats[:n].copy(),
                   frames=frames[:n].reshape(n, 3, 3).copy())
        if loc_out is not None:
            out["local"] = loc_out
        if Dout is not None:
            out["D_lab"] = Dout
        return out

    def mlp_grad(self, type_: int, X, Y):
        """Test hook: (loss, params, grads) of the network on X[n, 96], Y[n, width]."""
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        loss = np.zeros(1)
        P = np.zeros(self.nparam, np.float32)
        G = np.zeros(self.nparam, np.float32)
        _check(load().pimd_guess_mlp_grad(self.handle, X.shape[0], int(type_), _fp(X), _fp(Y), _dp(loss), _fp(P),
                                          _fp(G)), "pimd_guess_mlp_grad")
        return float(loss[0]), P, G

    def __del__(self):
        try:
            if self.handle:
                load().pimd_guess_destroy(self.handle)
        except Exception:
            pass
