"""Build the CUDA library `_build/libpimdgb.so` for sm_103a.

Steps: run the ERI code generator (csrc/gen_eri.py) into `_build/gen`, write
one translation unit per quartet class (Fock build + Schwarz, and gradient)
plus a dispatch table, compile every unit with nvcc in parallel, link a shared
library. Object files are cached by a hash of their inputs and flags.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import importlib.util
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
OBJ = os.path.join(BUILD, "obj")
LIB = os.path.join(BUILD, "libpimdgb.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-warn-spills", "-w", "-I" + CSRC, "-I" + GEN, "-I" + INCLUDE]
HAND_WRITTEN = ["onee.cu", "linalg.cu", "scf.cu", "peaks.cu", "guess.cu"]
# Units whose straight-line kernels ptxas -O3 allocates with 32 registers and
# tens of kilobytes of local-memory spills per thread (the FP64 (dd|dp) Fock
# kernel: 94 KB of spill stores); -O1 keeps 255 registers and spills 3-5x
# less (measured with -Xptxas -v for every unit at both levels).
PTXAS_O1 = {"tu_eri_dddp", "tu_eri_ddpp", "tu_eri_dpdp", "tu_grad_ddps", "tu_grad_ddss", "tu_grad_dpds",
            "tu_grad_dppp", "tu_grad_dpps", "tu_grad_dsds", "tu_grad_dspp", "tu_grad_pppp"}


def nvcc_path():
    env = os.environ.get("NVCC")
    if env:
        return env
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _gen_module():
    spec = importlib.util.spec_from_file_location("gen_eri", os.path.join(CSRC, "gen_eri.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _write(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


def _coop_upload_code(nm, grad, g):
    """C++ lines defining coop_tape_<nm>(CoopTape&, int& W, size_t& bytes,
    int& Wf, size_t& bytesf): uploads the class's tape once per device and
    sizes the FP64 and FP32 launches (warps per block, shared memory)."""
    pre = f"coop{'g' if grad else 'e'}_{nm}"
    st = f"Coop{'G' if grad else 'E'}_{nm}"
    c = [cl for cl in g.classes() if g.cls_name(cl) == nm][0]
    hr = g.grad_hrrs(c) if grad else [("E", c, "acc")]
    la, lb, lc, ld = c
    nc4 = g.ncart(la) * g.ncart(lb) * g.ncart(lc) * g.ncart(ld)
    kernel = (f"grad2e_coop_kernel<{la}, {lb}, {lc}, {ld}" if grad else f"jk_coop_kernel<{la}, {lb}, {lc}, {ld}")
    lines = ["static CoopTape g_coop[64];", "static bool g_coop_up[64];",
             "template <typename T> static const T* coop_copy(const T* h, size_t n)",
             "{", "    T* d = nullptr;", "    cudaMalloc(&d, n * sizeof(T));",
             "    cudaMemcpy(d, h, n * sizeof(T), cudaMemcpyHostToDevice);", "    return d;", "}",
             f"static void coop_tape_{nm}(CoopTape& t, int& W, size_t& bytes, int& Wf, size_t& bytesf)", "{",
             "    int dev = 0;", "    cudaGetDevice(&dev);",
             "    // warps per block (1..4): the count that puts the most warps on an SM",
             "    // within its shared memory (one workspace per block)",
             f"    W = coop_best_warps({st}::NACC, {st}::NWORK, {st}::L, {nc4}, sizeof(double));",
             f"    bytes = (size_t)coop_block_elems({st}::NACC, {st}::NWORK, {st}::L, {nc4}, 32 * W) * sizeof(double);",
             f"    Wf = coop_best_warps({st}::NACC, {st}::NWORK, {st}::L, {nc4}, sizeof(float));",
             f"    bytesf = (size_t)coop_block_elems({st}::NACC, {st}::NWORK, {st}::L, {nc4}, 32 * Wf) * sizeof(float);",
             "    if (dev >= 0 && dev < 64 && !g_coop_up[dev]) {",
             "        CoopTape c{};",
             f"        c.vrr = coop_copy({pre}_vrr, sizeof({pre}_vrr) / sizeof(int));",
             f"        c.vrr_lv = coop_copy({pre}_vrr_lv, sizeof({pre}_vrr_lv) / sizeof(int));",
             f"        c.acc = coop_copy({pre}_acc, sizeof({pre}_acc) / sizeof(int));",
             f"        c.nvlev = {st}::NVLEV;", f"        c.naccop = {st}::NACCOP;",
             f"        c.nhrr = {len(hr)};",
             f"        c.L = {st}::L;", f"        c.NACC = {st}::NACC;", f"        c.F0 = {st}::F0;",
             f"        c.NWORK = {st}::NWORK;"]
    for k, (hname, cls_, src) in enumerate(hr):
        pos = {"A": 0, "B": 1, "C": 2, "E": 0}[hname[0]]
        up = 1 if hname.endswith("p") or hname == "E" else 0
        lines += [f"        c.hrr[{k}] = coop_copy({pre}_hrr{hname}, sizeof({pre}_hrr{hname}) / sizeof(int));",
                  f"        c.hrr_lv[{k}] = coop_copy({pre}_hrr{hname}_lv, sizeof({pre}_hrr{hname}_lv) / sizeof(int));",
                  f"        c.nhlev[{k}] = (int)(sizeof({pre}_hrr{hname}_lv) / sizeof(int)) - 1;",
                  f"        c.out[{k}] = coop_copy({pre}_out{hname}, sizeof({pre}_out{hname}) / sizeof(int));",
                  f"        c.hpos[{k}] = {pos};", f"        c.hup[{k}] = {up};"]
    lines += ["        g_coop[dev] = c;", "        g_coop_up[dev] = true;",
              f"        cudaFuncSetAttribute({kernel}, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);",
              f"        cudaFuncSetAttribute({kernel}, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytesf);",
              f"        cudaFuncSetAttribute({kernel}, double>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);",
              f"        cudaFuncSetAttribute({kernel}, float>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);",
              "    }", "    t = g_coop[dev];", "}"]
    return lines


def generate_sources():
    """Generated headers + per-class translation units + dispatch. Returns the
    list of generated .cu files."""
    g = _gen_module()
    os.makedirs(GEN, exist_ok=True)
    stats = g.generate(GEN)
    heavy = {s[0]: s[6] for s in stats}
    coop_e = {s[0]: s[7] for s in stats}
    coop_g = {s[0]: s[8] for s in stats}
    straight_e = {s[0]: s[9] for s in stats}
    classes = g.classes()
    names = [g.cls_name(c) for c in classes]
    tus = []
    for c, nm in zip(classes, names):
        la, lb, lc, ld = c
        same = (la, lb) == (lc, ld)
        e = ['#include "coop_kernels.cuh"', '#include "internal.h"', f'#include "eri_{nm}.cuh"']
        if coop_e[nm]:
            e.append(f'#include "coope_{nm}.cuh"')
        e.append("namespace pimd {")
        if coop_e[nm]:
            e += _coop_upload_code(nm, False, g)
        # bs > 0: straight-line kernel with bs threads per block; bs == 0: the
        # cooperative tape kernel
        e += [f"void launch_jk_{nm}(const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles,",
              "                     const double* D, const float* Df, double* G, const double* boys,",
              "                     const float* boysf, double tau, double fp32_tau, const double* Dsh,",
              "                     unsigned long long* cnt, int bs, double tp, double fxs, cudaStream_t st)",
              "{",
              "    if (ntiles <= 0) return;",
              "    const double split = fp32_tau > tau ? fp32_tau : tau;"]
        if coop_e[nm]:
            e += [f"    if (bs == 0{'' if straight_e[nm] else ' || true'}) {{",
                  "        CoopTape t; int W, Wf; size_t bytes, bytesf;",
                  f"        coop_tape_{nm}(t, W, bytes, Wf, bytesf);",
                  f"        jk_coop_kernel<{la}, {lb}, {lc}, {ld}, double><<<ntiles, 32 * W, bytes, st>>>(P, S, R, tiles,",
                  "            D, G, boys, split, 1e300, Dsh, cnt, t, tp, fxs);",
                  "        if (fp32_tau > tau)",
                  f"            jk_coop_kernel<{la}, {lb}, {lc}, {ld}, float><<<ntiles, 32 * Wf, bytesf, st>>>(P, S, R,",
                  "                tiles, Df, G, boysf, tau, fp32_tau, Dsh, cnt + 2, t, tp, fxs);",
                  "        return;",
                  "    }"]
        if straight_e[nm]:
            e += ["    const int b = bs > 0 ? bs : 128;",
                  f"    jk_kernel<Cls_{nm}, double><<<ntiles, b, 0, st>>>(P, S, R, tiles, D, G, boys, split, 1e300, Dsh, cnt,",
                  "                                                      tp, fxs);",
                  "    if (fp32_tau > tau)",
                  f"        jk_kernel<Cls_{nm}, float><<<ntiles, b, 0, st>>>(P, S, R, tiles, Df, G, boysf, tau, fp32_tau, Dsh,",
                  "                                                       cnt + 2, tp, fxs);"]
        e.append("}")
        if same:
            e += [f"void launch_schwarz_{nm}(const Pairs& P, const Shells& S, const int* list, int n,",
                  "                          const double* boys, double* Q, cudaStream_t st)",
                  "{",
                  f"    if (n > 0) schwarz_kernel<Cls_{nm}><<<(n + 127) / 128, 128, 0, st>>>(P, S, list, n, boys, Q);",
                  "}",
                  f"void launch_prim_schwarz_{nm}(const Pairs& P, const Shells& S, const int* list, int n,",
                  "                               const double* boys, double* pp, float* qp, float* qg, cudaStream_t st)",
                  "{",
                  f"    if (n > 0) prim_schwarz_kernel<Cls_{nm}><<<(n + 127) / 128, 128, 0, st>>>(P, S, list, n, boys, pp, qp, qg);",
                  "}"]
        e.append("}  // namespace pimd\n")
        p = os.path.join(GEN, f"tu_eri_{nm}.cu")
        _write(p, "\n".join(e))
        tus.append(p)
        gl = ['#include "coop_kernels.cuh"', '#include "internal.h"', f'#include "grad_{nm}.cuh"']
        if coop_g[nm]:
            gl.append(f'#include "coopg_{nm}.cuh"')
        gl.append("namespace pimd {")
        if coop_g[nm]:
            gl += _coop_upload_code(nm, True, g)
            gl.append(f"void grad2e_upload_{nm}() {{ CoopTape t; int W, Wf; size_t b, bf; coop_tape_{nm}(t, W, b, Wf, bf); }}")
        else:
            gl.append(f"void grad2e_upload_{nm}() {{}}")
        # variant 0: cooperative tape kernel, 1: straight-line kernel with bs threads
        gl += [f"void launch_grad2e_{nm}(const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles,",
               "                        const double* D, double* grad, const double* boys, const float* boysf,",
               "                        double tau, double fp32_tau, const double* Dsh, unsigned long long* cnt,",
               "                        int variant, int bs, double tp, double fxs, cudaStream_t st)",
               "{",
               "    if (ntiles <= 0) return;",
               "    const double split = fp32_tau > tau ? fp32_tau : tau;"]
        if coop_g[nm]:
            gl += [f"    if (variant == 0{' || true' if heavy[nm] else ''}) {{",
                   "        CoopTape t; int W, Wf; size_t bytes, bytesf;",
                   f"        coop_tape_{nm}(t, W, bytes, Wf, bytesf);",
                   f"        grad2e_coop_kernel<{la}, {lb}, {lc}, {ld}, double><<<ntiles, 32 * W, bytes, st>>>(P, S, R,",
                   "            tiles, D, grad, boys, split, 1e300, Dsh, cnt, t, tp, fxs);",
                   "        if (fp32_tau > tau)",
                   f"            grad2e_coop_kernel<{la}, {lb}, {lc}, {ld}, float><<<ntiles, 32 * Wf, bytesf, st>>>(P, S,",
                   "                R, tiles, D, grad, boysf, tau, fp32_tau, Dsh, cnt + 2, t, tp, fxs);",
                   "        return;",
                   "    }"]
        if not heavy[nm]:
            gl += ["    const int b = bs > 0 ? bs : 128;",
                   f"    grad2e_kernel<GCls_{nm}, double><<<ntiles, b, 0, st>>>(P, S, R, tiles, D, grad, boys, split, 1e300, Dsh,",
                   "                                                            cnt, tp, fxs);",
                   "    if (fp32_tau > tau)",
                   f"        grad2e_kernel<GCls_{nm}, float><<<ntiles, b, 0, st>>>(P, S, R, tiles, D, grad, boysf, tau, fp32_tau,",
                   "                                                           Dsh, cnt + 2, tp, fxs);"]
        gl.append("}")
        gl.append("}  // namespace pimd\n")
        p = os.path.join(GEN, f"tu_grad_{nm}.cu")
        _write(p, "\n".join(gl))
        tus.append(p)
    # dispatch
    d = ['#include "internal.h"', "namespace pimd {"]
    sig_jk = ("const Pairs&, const Shells&, const Reps&, const Tile*, int, const double*, const float*, double*, "
              "const double*, const float*, double, double, const double*, unsigned long long*, int, double, "
              "double, cudaStream_t")
    sig_sw = "const Pairs&, const Shells&, const int*, int, const double*, double*, cudaStream_t"
    sig_psw = "const Pairs&, const Shells&, const int*, int, const double*, double*, float*, float*, cudaStream_t"
    sig_g = ("const Pairs&, const Shells&, const Reps&, const Tile*, int, const double*, double*, const double*, "
             "const float*, double, double, const double*, unsigned long long*, int, int, double, double, cudaStream_t")
    for c, nm in zip(classes, names):
        d.append(f"void launch_jk_{nm}({sig_jk});")
        if (c[0], c[1]) == (c[2], c[3]):
            d.append(f"void launch_schwarz_{nm}({sig_sw});")
            d.append(f"void launch_prim_schwarz_{nm}({sig_psw});")
        d.append(f"void launch_grad2e_{nm}({sig_g});")
        d.append(f"void grad2e_upload_{nm}();")
    d.append(f"int n_class_pairs() {{ return {len(classes)}; }}")
    d.append("void class_pair_ls(int cp, int* la, int* lb, int* lc, int* ld)")
    d.append("{")
    d.append("    static const int t[][4] = {" + ", ".join("{%d, %d, %d, %d}" % c for c in classes) + "};")
    d.append("    *la = t[cp][0]; *lb = t[cp][1]; *lc = t[cp][2]; *ld = t[cp][3];")
    d.append("}")
    flops = {s[0]: s[2] for s in stats}
    d.append("long long class_vrr_flops(int cp)")
    d.append("{")
    # per primitive quartet: the generated recursion's operations (an FMA
    # counts 2) plus the set-up of prim_quartet (25) and the Boys function
    # (17 for the Taylor step and prefactor; for L > 0 also 16 for e^{-T} and
    # 3 per order of the downward recursion)
    d.append("    static const long long t[] = {" + ", ".join(str(flops[nm] + 42 + (16 + 3 * sum(c) if sum(c) else 0))
                                                        for c, nm in zip(classes, names)) + "};")
    d.append("    return t[cp];")
    d.append("}")
    gflops = {s[0]: s[5] for s in stats}
    d.append("long long class_grad_flops(int cp)")
    d.append("{")
    # per primitive quartet of the gradient: the generated recursion to order
    # L + 1 with its four accumulated sets, the same set-up (42) and the Boys
    # function to order L + 1 (16 + 3 (L + 1))
    d.append("    static const long long t[] = {" + ", ".join(str(gflops[nm] + 42 + 16 + 3 * (sum(c) + 1))
                                                        for c, nm in zip(classes, names)) + "};")
    d.append("    return t[cp];")
    d.append("}")
    d.append(f"typedef void (*JkFn)({sig_jk});")
    d.append("static const JkFn jk_tab[] = {" + ", ".join(f"launch_jk_{nm}" for nm in names) + "};")
    d.append("void launch_jk(int cp, const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles, "
             "const double* D, const float* Df, double* G, const double* boys, const float* boysf, double tau, "
             "double fp32_tau, const double* Dsh, unsigned long long* cnt, int bs, double tau_prim, double fxs, "
             "cudaStream_t st)")
    d.append("{ jk_tab[cp](P, S, R, tiles, ntiles, D, Df, G, boys, boysf, tau, fp32_tau, Dsh, cnt, bs, tau_prim, fxs, st); }")
    for fn, tab in (("class_pair_coop", coop_e), ("class_pair_straight", straight_e), ("grad_pair_coop", coop_g),
                    ("grad_pair_straight", {nm: not heavy[nm] for nm in names})):
        d.append(f"bool {fn}(int cp)")
        d.append("{")
        d.append("    static const bool t[] = {" + ", ".join("true" if tab[nm] else "false" for nm in names) + "};")
        d.append("    return t[cp];")
        d.append("}")
    same = [nm for c, nm in zip(classes, names) if (c[0], c[1]) == (c[2], c[3])]
    d.append(f"typedef void (*SwFn)({sig_sw});")
    d.append("static const SwFn sw_tab[] = {" + ", ".join(f"launch_schwarz_{nm}" for nm in same) + "};")
    d.append("void launch_schwarz(int X, const Pairs& P, const Shells& S, const int* list, int n, const double* boys, "
             "double* Q, cudaStream_t st)")
    d.append("{ sw_tab[X](P, S, list, n, boys, Q, st); }")
    d.append(f"typedef void (*PswFn)({sig_psw});")
    d.append("static const PswFn psw_tab[] = {" + ", ".join(f"launch_prim_schwarz_{nm}" for nm in same) + "};")
    d.append("void launch_prim_schwarz(int X, const Pairs& P, const Shells& S, const int* list, int n, "
             "const double* boys, double* pp, float* qp, float* qg, cudaStream_t st)")
    d.append("{ psw_tab[X](P, S, list, n, boys, pp, qp, qg, st); }")
    d.append(f"typedef void (*GFn)({sig_g});")
    d.append("static const GFn g_tab[] = {" + ", ".join(f"launch_grad2e_{nm}" for nm in names) + "};")

    d.append("void launch_grad2e(int cp, const Pairs& P, const Shells& S, const Reps& R, const Tile* tiles, int ntiles, "
             "const double* D, double* grad, const double* boys, const float* boysf, double tau, double fp32_tau, "
             "const double* Dsh, unsigned long long* cnt, int variant, int bs, double tau_prim, double fxs, "
             "cudaStream_t st)")
    d.append("{ g_tab[cp](P, S, R, tiles, ntiles, D, grad, boys, boysf, tau, fp32_tau, Dsh, cnt, variant, bs, tau_prim, "
             "fxs, st); }")
    d.append("void grad2e_tapes_upload() {")
    for nm in names:
        d.append(f"    grad2e_upload_{nm}();")
    d.append("}")
    d.append("}  // namespace pimd\n")
    p = os.path.join(GEN, "tu_dispatch.cu")
    _write(p, "\n".join(d))
    tus.append(p)
    return tus


def _deps_hash(src, extra):
    h = hashlib.sha1()
    h.update(" ".join(ARCH + FLAGS).encode())
    with open(src, "rb") as fh:
        h.update(fh.read())
    for dep in extra:
        with open(dep, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _compile(args):
    src, obj, digest = args
    stamp = obj + ".sha1"
    if os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == digest:
        return src, 0.0, ""
    import time
    t = time.time()
    extra = ["-Xptxas", "-O1"] if os.path.basename(src)[:-3] in PTXAS_O1 else []
    cmd = [nvcc_path()] + ARCH + FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return src, time.time() - t, r.stderr


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    tus = generate_sources()
    common = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    common.append(os.path.join(INCLUDE, "pimdgb.h"))
    work = []
    for f in HAND_WRITTEN:
        src = os.path.join(CSRC, f)
        work.append((src, os.path.join(OBJ, f + ".o"), _deps_hash(src, common)))
    for src in tus:
        base = os.path.basename(src)
        deps = list(common)
        if base.startswith("tu_eri_") or base.startswith("tu_grad_"):
            nm = base.split("_")[-1][:-3]
            kind = "eri" if base.startswith("tu_eri_") else "grad"
            deps.append(os.path.join(GEN, f"{kind}_{nm}.cuh"))
            for tp in (os.path.join(GEN, f"grad_tape_{nm}.cuh"), os.path.join(GEN, f"coope_{nm}.cuh"),
                       os.path.join(GEN, f"coopg_{nm}.cuh")):
                if os.path.exists(tp):
                    deps.append(tp)
        extra = "ptxas-O1" if base[:-3] in PTXAS_O1 else ""
        work.append((src, os.path.join(OBJ, base + ".o"), _deps_hash(src, deps) + extra))
    if force:
        for _, obj, _ in work:
            if os.path.exists(obj + ".sha1"):
                os.remove(obj + ".sha1")
    # largest units first so that the long ones start early
    work.sort(key=lambda w: -os.path.getsize(w[0]) - sum(os.path.getsize(os.path.join(GEN, x))
                                                            for x in os.listdir(GEN)
                                                            if x.endswith(".cuh") and x[:-4].split("_")[-1]
                                                            == os.path.basename(w[0])[:-3].split("_")[-1]))
    jobs = jobs or max(1, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(jobs) as ex:
        for src, dt, err in ex.map(_compile, work):
            if verbose and dt > 0:
                print(f"  {os.path.basename(src)}: {dt:.1f}s", flush=True)
    objs = [w[1] for w in work]
    link_digest = hashlib.sha1("".join(open(o + ".sha1").read() for o in objs).encode()).hexdigest()
    stamp = LIB + ".sha1"
    if not (os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == link_digest):
        cmd = [nvcc_path()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
        with open(stamp, "w") as fh:
            fh.write(link_digest)
    return LIB


if __name__ == "__main__":
    import time
    t0 = time.time()
    print(build(force="--force" in sys.argv, verbose=True), f"{time.time() - t0:.1f}s")
