"""C-ABI library: it builds, loads without a GPU and exports every entry
point that include/pimdgb.h declares; host-side argument checks."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1601_02713_gb300 import build as B
from paper_1601_02713_gb300 import inputs, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return native.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "pimdgb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["pimd_bo_forces", "string_images_forces", "pimd_ctx_create", "pimd_basis_create", "pimd_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_strerror_and_defaults(lib):
    assert native.strerror(0) == "ok"
    assert "invalid" in native.strerror(-1)
    o = native.scf_opts()
    assert o.struct_size == ctypes.sizeof(native.PimdScfOpts)
    assert o.conv_energy == 1e-10 and o.conv_error == 1e-8 and o.schwarz_tau == 1e-12
    assert o.max_iter == 64 and o.diis_size == 8 and o.want_gradient == 1


def test_basis_create_and_validation(lib):
    bas = inputs.basis_set("split_spd")
    b = native.Basis(bas)
    assert b.nbf([8, 1, 1]) == 24
    assert b.nbf([6] * 9 + [1] * 12 + [8]) == 200
    with pytest.raises(native.PimdError):
        b.nbf([7])  # nitrogen is not in the basis
    Zs, nsh, sl, snp, ex, co = inputs.basis_arrays(bas)
    h = ctypes.c_void_p()
    bad_l = sl.copy()
    bad_l[0] = 3
    rc = lib.pimd_basis_create(ctypes.byref(h), len(Zs), native._ip(Zs), native._ip(nsh), native._ip(bad_l),
                               native._ip(snp), native._dp(ex), native._dp(co), 1)
    assert rc == native.PIMD_EINVAL
    bad_e = ex.copy()
    bad_e[2] = -1.0
    rc = lib.pimd_basis_create(ctypes.byref(h), len(Zs), native._ip(Zs), native._ip(nsh), native._ip(sl),
                               native._ip(snp), native._dp(bad_e), native._dp(co), 1)
    assert rc == native.PIMD_EINVAL
    rc = lib.pimd_basis_create(ctypes.byref(h), len(Zs), native._ip(Zs), native._ip(nsh), native._ip(sl),
                               native._ip(snp), native._dp(ex), native._dp(co), 0)
    assert rc == native.PIMD_EINVAL


def test_forces_reject_null_context(lib):
    Z = np.array([8, 1, 1], np.int32)
    X = np.zeros((1, 3, 3))
    E = np.zeros(1)
    G = np.zeros((1, 3, 3))
    rc = lib.pimd_bo_forces(None, 1, 3, native._ip(Z), native._dp(X), None, None, native._dp(E), native._dp(G), None)
    assert rc == native.PIMD_EINVAL


def test_diagnostics_reject_null_context(lib):
    """The per-call records answer PIMD_EINVAL for a missing context or a
    negative count instead of touching memory (no GPU involved)."""
    st = native.PimdStats()
    assert lib.pimd_last_stats(None, ctypes.byref(st)) == native.PIMD_EINVAL
    assert lib.pimd_last_trace(None, 0, 0, None, None, None) == native.PIMD_EINVAL
    assert lib.pimd_last_fock_times(None, 0, None, None) == native.PIMD_EINVAL
    assert lib.pimd_last_fock_times(None, -1, None, None) == native.PIMD_EINVAL


def test_generated_sources_are_deterministic():
    g = B._gen_module()
    import tempfile
    with tempfile.TemporaryDirectory() as d1, tempfile.TemporaryDirectory() as d2:
        g.generate(d1)
        g.generate(d2)
        for f in sorted(os.listdir(d1)):
            assert open(os.path.join(d1, f)).read() == open(os.path.join(d2, f)).read(), f


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the offsets and sizes the C
    compiler gives the header's structs (a header/binding drift would
    silently misread options or statistics)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"pimd_scf_opts": native.PimdScfOpts, "pimd_info": native.PimdInfo, "pimd_stats": native.PimdStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "pimdgb.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_eigensolver_wrappers_reject_bad_tensors_without_a_launch(lib):
    """The binding checks dtype, contiguity, shapes and device of the
    eigensolver's tensors before calling into the library: every case here
    is refused with PIMD_EINVAL (CPU tensors, so a call that got through would
    fail on the device check or in the library, never silently)."""
    torch = pytest.importorskip("torch")
    n, nmat = 6, 2
    A = torch.zeros(nmat, n, n, dtype=torch.float64)
    V = torch.zeros(nmat, n, n, dtype=torch.float64)
    w = torch.zeros(nmat, n, dtype=torch.float64)
    bad = [
        (A.float(), V, w),                                   # float32 input
        (A, V.float(), w),                                   # float32 output
        (A.transpose(1, 2), V, w),                           # strided (non-contiguous) input
        (torch.zeros(nmat, n, n + 1, dtype=torch.float64), V, w),   # A not square
        (A, torch.zeros(nmat, n - 1, n, dtype=torch.float64), w),   # V too small
        (A, V, torch.zeros(nmat, n - 1, dtype=torch.float64)),      # evals too small
        (A, V, torch.zeros(nmat - 1, n, dtype=torch.float64)),      # fewer eigenvalue rows than matrices
        (torch.zeros(0, n, n, dtype=torch.float64), V[:0], w[:0]),  # empty batch
        (A, V, w),                                           # valid shapes, but host tensors
    ]
    for args in bad:
        assert not native.eigh_args_ok(*args)
        assert native.pimd_eigh_noalloc(*args) == native.PIMD_EINVAL
        with pytest.raises(native.PimdError) as ei:
            native.pimd_eigh_dev(None, *args)
        assert ei.value.code == native.PIMD_EINVAL


def test_noalloc_size_limits_checked_before_any_device_call(lib):
    """pimd_eigh_noalloc refuses sizes beyond its fixed workspace (n <= 768,
    nmat <= 1024, nmat * n * n <= 2,097,152) before it touches the device:
    each case is one past a limit (or empty, or a null pointer), and the
    pointers are never dereferenced. The cases at the limits run against
    real device buffers in the GPU tests."""
    p = ctypes.c_void_p(16)
    f = lib.pimd_eigh_noalloc
    assert f(4, 768, p, p, p, None) == native.PIMD_EINVAL          # 2,359,296 doubles
    assert f(1025, 2, p, p, p, None) == native.PIMD_EINVAL         # one descriptor too many
    assert f(1, 769, p, p, p, None) == native.PIMD_EINVAL          # column longer than the solver holds
    assert f(0, 4, p, p, p, None) == native.PIMD_EINVAL
    assert f(2, 0, p, p, p, None) == native.PIMD_EINVAL
    assert f(2, 4, None, p, p, None) == native.PIMD_EINVAL
