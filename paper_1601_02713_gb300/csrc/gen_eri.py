"""Code generator for the shell-quartet ERI kernels (Obara-Saika vertical
recursion + Head-Gordon-Pople horizontal recursion).

For every class (la lb | lc ld) with la >= lb, lc >= ld it emits straight-line
device code:

* `vrr_<cls>`: per primitive quartet, builds the target set of
  [e0|f0]^(0) from [00|00]^(m) = Theta F_m(T) with the two Obara-Saika rules
  (Obara & Saika, J. Chem. Phys. 84, 3963 (1986); Head-Gordon & Pople,
  J. Chem. Phys. 89, 5777 (1988)):
    [e+1_i,0|00]^(m) = PA_i [e0|00]^(m) + WP_i [e0|00]^(m+1)
                       + e_i/(2p) ([e-1_i,0|00]^(m) - rho/p [e-1_i,0|00]^(m+1))
    [e0|f+1_i,0]^(m) = QC_i [e0|f0]^(m) + WQ_i [e0|f0]^(m+1)
                       + f_i/(2q) ([e0|f-1_i,0]^(m) - rho/q [e0|f-1_i,0]^(m+1))
                       + e_i/(2(p+q)) [e-1_i,0|f0]^(m+1)
  and adds them (optionally times weights) into contracted accumulators;
* `hrr_<cls>`: after contraction, the horizontal rules
    (a, b+1_i| = (a+1_i, b| + AB_i (a, b|      (bra)
    |c, d+1_i) = |c+1_i, d) + CD_i |c, d)      (ket)
  giving the Cartesian block (ab|cd).

Only intermediates that a target needs are emitted (demand-driven, memoised).
The generated header is written to the build directory by `build()`; the
generator is pure Python and deterministic.
"""
from __future__ import annotations

import itertools
import sys

LMAX = 2  # s, p, d shells


def carts(l):
    """Cartesian components (lx, ly, lz), lx = l..0, ly = l-lx..0."""
    out = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            out.append((lx, ly, l - lx - ly))
    return out


def ncart(l):
    return (l + 1) * (l + 2) // 2


def sub(v, i, k=1):
    w = list(v)
    w[i] -= k
    return tuple(w)


def add(v, i, k=1):
    w = list(v)
    w[i] += k
    return tuple(w)


def pick_dir(v):
    """Direction to decrement: the largest component, ties to the lowest axis."""
    m = max(v)
    return v.index(m)


class VRRGen:
    """Demand-driven [e0|f0]^(m) generator."""

    def __init__(self):
        self.memo = {}
        self.lines = []
        self.n = 0

    def get(self, e, f, m):
        if min(e) < 0 or min(f) < 0:
            return None
        key = (e, f, m)
        if key in self.memo:
            return self.memo[key]
        if sum(e) == 0 and sum(f) == 0:
            name = f"F{m}"
            self.memo[key] = name
            return name
        if sum(f) > 0:
            i = pick_dir(f)
            f1 = sub(f, i)
            terms = []
            t1 = self.get(e, f1, m)
            t2 = self.get(e, f1, m + 1)
            terms.append(f"QC{i}*{t1}")
            terms.append(f"WQ{i}*{t2}")
            if f1[i] > 0:
                f2 = sub(f1, i)
                t3 = self.get(e, f2, m)
                t4 = self.get(e, f2, m + 1)
                k = f1[i]
                terms.append(f"R({k})*(o2q*{t3} - o2qr*{t4})" if k > 1 else f"(o2q*{t3} - o2qr*{t4})")
            if e[i] > 0:
                t5 = self.get(sub(e, i), f1, m + 1)
                k = e[i]
                terms.append(f"R({k})*o2pq*{t5}" if k > 1 else f"o2pq*{t5}")
        else:
            i = pick_dir(e)
            e1 = sub(e, i)
            t1 = self.get(e1, f, m)
            t2 = self.get(e1, f, m + 1)
            terms = [f"PA{i}*{t1}", f"WP{i}*{t2}"]
            if e1[i] > 0:
                e2 = sub(e1, i)
                t3 = self.get(e2, f, m)
                t4 = self.get(e2, f, m + 1)
                k = e1[i]
                terms.append(f"R({k})*(o2p*{t3} - o2pr*{t4})" if k > 1 else f"(o2p*{t3} - o2pr*{t4})")
        name = f"v{self.n}"
        self.n += 1
        self.lines.append(f"const R {name} = " + " + ".join(terms) + ";")
        self.memo[key] = name
        return name


def level_range(lo, hi):
    out = []
    for l in range(max(lo, 0), hi + 1):
        out += carts(l)
    return out


def gen_vrr(name, Ltot, acc_sets, grad_sig=False):
    """acc_sets: list of (acc_name, e_lo, e_hi, f_lo, f_hi, weight_expr or None).
    Emits a device function adding [e0|f0]^(0) for every listed (e, f) into
    acc_name[idx] (times weight)."""
    g = VRRGen()
    body_acc = []
    for acc, elo, ehi, flo, fhi, w in acc_sets:
        es = level_range(elo, ehi)
        fs = level_range(flo, fhi)
        for ie, e in enumerate(es):
            for jf, f in enumerate(fs):
                v = g.get(e, f, 0)
                idx = ie * len(fs) + jf
                body_acc.append(f"{acc}[{idx}] += {w}*{v};" if w else f"{acc}[{idx}] += {v};")
    if grad_sig:
        args = "R* __restrict__ accU, R* __restrict__ accA, R* __restrict__ accB, R* __restrict__ accC, R wa, R wb, R wc"
    else:
        args = "R* __restrict__ acc"
    hdr = (f"template <typename R>\nstatic __device__ __forceinline__ void {name}(const R* __restrict__ Fm, "
           f"R PA0, R PA1, R PA2, R WP0, R WP1, R WP2, R QC0, R QC1, R QC2, R WQ0, R WQ1, R WQ2, "
           f"R o2p, R o2pr, R o2q, R o2qr, R o2pq, {args})\n{{\n")
    used_m = sorted({int(k[2]) for k in g.memo if sum(k[0]) == 0 and sum(k[1]) == 0})
    pre = "".join(f"    const R F{m} = Fm[{m}];\n" for m in used_m)
    body = "\n".join("    " + l for l in g.lines + body_acc)
    nflop = sum(l.count("*") + l.count("+") + l.count(" - ") for l in g.lines) + len(body_acc) * 2
    return hdr + pre + body + "\n}\n", len(g.lines), nflop


class HRRGen:
    """Demand-driven (ab|cd) from contracted (e0|f0)."""

    def __init__(self, es, fs, src):
        self.eidx = {e: i for i, e in enumerate(es)}
        self.fidx = {f: i for i, f in enumerate(fs)}
        self.nf = len(fs)
        self.src = src
        self.memo = {}
        self.lines = []
        self.n = 0

    def get(self, a, b, c, d):
        key = (a, b, c, d)
        if key in self.memo:
            return self.memo[key]
        if sum(b) == 0 and sum(d) == 0:
            name = f"{self.src}[{self.eidx[a] * self.nf + self.fidx[c]}]"
            self.memo[key] = name
            return name
        if sum(d) > 0:
            i = pick_dir(d)
            d1 = sub(d, i)
            t1 = self.get(a, b, add(c, i), d1)
            t2 = self.get(a, b, c, d1)
            expr = f"{t1} + CD{i}*{t2}"
        else:
            i = pick_dir(b)
            b1 = sub(b, i)
            t1 = self.get(add(a, i), b1, c, d)
            t2 = self.get(a, b1, c, d)
            expr = f"{t1} + AB{i}*{t2}"
        name = f"h{self.n}"
        self.n += 1
        self.lines.append(f"const R {name} = {expr};")
        self.memo[key] = name
        return name


def gen_hrr(name, la, lb, lc, ld, elo, ehi, flo, fhi):
    """Emit a function writing the Cartesian block out[((a*nb+b)*nc+c)*nd+d]
    of class (la lb|lc ld) from src = contracted (e0|f0), e in [elo, ehi],
    f in [flo, fhi] (levels)."""
    es = level_range(elo, ehi)
    fs = level_range(flo, fhi)
    g = HRRGen(es, fs, "src")
    outs = []
    A, B, C, D = carts(la), carts(lb), carts(lc), carts(ld)
    for ia, a in enumerate(A):
        for ib, b in enumerate(B):
            for ic, c in enumerate(C):
                for id_, d in enumerate(D):
                    v = g.get(a, b, c, d)
                    idx = ((ia * len(B) + ib) * len(C) + ic) * len(D) + id_
                    outs.append(f"out[{idx}] = {v};")
    hdr = (f"template <typename R>\nstatic __device__ __forceinline__ void {name}(const R* __restrict__ src, "
           f"R AB0, R AB1, R AB2, R CD0, R CD1, R CD2, R* __restrict__ out)\n{{\n")
    body = "\n".join("    " + l for l in g.lines + outs)
    return hdr + body + "\n}\n", len(g.lines)


def classes():
    out = []
    pairs = [(la, lb) for la in range(LMAX + 1) for lb in range(la + 1)]
    for i, (la, lb) in enumerate(pairs):
        for (lc, ld) in pairs[: i + 1]:
            out.append((la, lb, lc, ld))
    return out


def cls_name(c):
    return "".join("spdfgh"[x] for x in c)


def n_range(lo, hi):
    return sum(ncart(l) for l in range(max(lo, 0), hi + 1))


def grad_sets(c):
    """Accumulator sets of the gradient VRR: unweighted U (for the lowered
    terms) and weighted by 2a, 2b, 2c (raised terms of centres A, B, C)."""
    la, lb, lc, ld = c
    sets = []
    if la + lb + lc > 0:
        sets.append(("accU", la - 1, la + lb, lc - 1 if lc > 0 else 0, lc + ld, None))
    sets += [("accA", la + 1, la + lb + 1, lc, lc + ld, "wa"),
             ("accB", la, la + lb + 1, lc, lc + ld, "wb"),
             ("accC", la, la + lb, lc + 1, lc + ld + 1, "wc")]
    return sets


def grad_hrrs(c):
    """(name, shifted class, source set) of the six derivative blocks."""
    la, lb, lc, ld = c
    out = [("Ap", (la + 1, lb, lc, ld), "accA"), ("Bp", (la, lb + 1, lc, ld), "accB"),
           ("Cp", (la, lb, lc + 1, ld), "accC")]
    if la > 0:
        out.append(("Am", (la - 1, lb, lc, ld), "accU"))
    if lb > 0:
        out.append(("Bm", (la, lb - 1, lc, ld), "accU"))
    if lc > 0:
        out.append(("Cm", (la, lb, lc - 1, ld), "accU"))
    return out


def set_range(sets, name):
    for s in sets:
        if s[0] == name:
            return s[1], s[2], s[3], s[4]
    raise KeyError(name)


# gradient classes whose straight-line code compiles quickly; the others run
# through the tape interpreter
HEAVY_GRAD_VRR_LINES = 900


def gen_tape(c):
    """Op tape for the gradient of class c (see grad_tape.cuh for the format).
    Returns (ops, nslot, slot layout dict)."""
    la, lb, lc, ld = c
    L = la + lb + lc + ld + 1
    sets = grad_sets(c)
    ops = []
    # slots 0..L: F_m (times the prefactor)
    slot = {}
    nxt = [L + 1]

    def new():
        v = nxt[0]
        nxt[0] += 1
        return v

    memo = {}

    def get(e, f, m):
        if min(e) < 0 or min(f) < 0:
            return -1
        key = (e, f, m)
        if key in memo:
            return memo[key]
        if sum(e) == 0 and sum(f) == 0:
            memo[key] = m
            return m
        if sum(f) > 0:
            i = pick_dir(f)
            f1 = sub(f, i)
            s1, s2 = get(e, f1, m), get(e, f1, m + 1)
            s3 = s4 = -1
            k1 = 0
            if f1[i] > 0:
                f2 = sub(f1, i)
                s3, s4 = get(e, f2, m), get(e, f2, m + 1)
                k1 = f1[i]
            s5 = -1
            k2 = 0
            if e[i] > 0:
                s5 = get(sub(e, i), f1, m + 1)
                k2 = e[i]
            d = new()
            ops.append((1, d, s1, s2, s3, s4, s5, i | (k1 << 4) | (k2 << 8)))
        else:
            i = pick_dir(e)
            e1 = sub(e, i)
            s1, s2 = get(e1, f, m), get(e1, f, m + 1)
            s3 = s4 = -1
            k1 = 0
            if e1[i] > 0:
                e2 = sub(e1, i)
                s3, s4 = get(e2, f, m), get(e2, f, m + 1)
                k1 = e1[i]
            d = new()
            ops.append((0, d, s1, s2, s3, s4, -1, i | (k1 << 4)))
        memo[key] = d
        return d

    acc_ops = []
    acc_base = {}
    wsel = {None: 0, "wa": 1, "wb": 2, "wc": 3}
    pending = []
    for name, elo, ehi, flo, fhi, w in sets:
        es, fs = level_range(elo, ehi), level_range(flo, fhi)
        for ie, e in enumerate(es):
            for jf, f in enumerate(fs):
                pending.append((name, ie * len(fs) + jf, get(e, f, 0), wsel[w]))
    for name, elo, ehi, flo, fhi, w in sets:
        n = n_range(elo, ehi) * n_range(flo, fhi)
        acc_base[name] = nxt[0]
        nxt[0] += n
    for name, idx, src, ws in pending:
        acc_ops.append((2, acc_base[name] + idx, src, -1, -1, -1, -1, ws))
    nvrr = len(ops)
    # HRRs of the shifted classes
    hrr_ops = []
    outs = {}
    for hname, (a_, b_, c_, d_), src in grad_hrrs(c):
        elo, ehi, flo, fhi = set_range(sets, src)
        es, fs = level_range(elo, ehi), level_range(flo, fhi)
        eidx = {e: i for i, e in enumerate(es)}
        fidx = {f: i for i, f in enumerate(fs)}
        hm = {}

        def hget(a, b, cc, dd):
            key = (a, b, cc, dd)
            if key in hm:
                return hm[key]
            if sum(b) == 0 and sum(dd) == 0:
                v = acc_base[src] + eidx[a] * len(fs) + fidx[cc]
                hm[key] = v
                return v
            if sum(dd) > 0:
                i = pick_dir(dd)
                d1 = sub(dd, i)
                s1, s2 = hget(a, b, add(cc, i), d1), hget(a, b, cc, d1)
                dst = new()
                hrr_ops.append((4, dst, s1, s2, -1, -1, -1, i))
            else:
                i = pick_dir(b)
                b1 = sub(b, i)
                s1, s2 = hget(add(a, i), b1, cc, dd), hget(a, b1, cc, dd)
                dst = new()
                hrr_ops.append((3, dst, s1, s2, -1, -1, -1, i))
            hm[key] = dst
            return dst

        o = []
        for a in carts(a_):
            for b in carts(b_):
                for cc in carts(c_):
                    for dd in carts(d_):
                        o.append(hget(a, b, cc, dd))
        outs[hname] = o
    return ops, acc_ops, hrr_ops, nxt[0], acc_base, outs, nvrr


HRR_NAMES = ["Ap", "Bp", "Cp", "Am", "Bm", "Cm"]


def write_if_changed(path, text):
    """Write text to path unless the file already holds exactly that text
    (keeps timestamps and build caches stable)."""
    import os
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return False
    with open(path, "w") as fh:
        fh.write(text)
    return True


def generate(outdir):
    """Write one header per class (energy VRR/HRR, gradient VRR/HRR or tape).
    Returns per-class statistics."""
    import os
    os.makedirs(outdir, exist_ok=True)
    stats = []
    tape_all = []
    for c in classes():
        la, lb, lc, ld = c
        nm = cls_name(c)
        L = la + lb + lc + ld
        parts = [f"// Generated by gen_eri.py for class ({nm[:2]}|{nm[2:]}).\n#pragma once\n\n"]
        code, nl, nfl = gen_vrr("vrr", L, [("acc", la, la + lb, lc, lc + ld, None)])
        hcode, nh = gen_hrr("hrr", la, lb, lc, ld, la, la + lb, lc, lc + ld)
        parts.append(f"struct Cls_{nm} {{\n  static constexpr int LA={la}, LB={lb}, LC={lc}, LD={ld}, L={L}, "
                     f"NE={n_range(la, la + lb)}, NF={n_range(lc, lc + ld)}, VRR_FLOPS={nfl};\n")
        parts.append(code)
        parts.append(hcode)
        parts.append("};\n")
        write_if_changed(os.path.join(outdir, f"eri_{nm}.cuh"), "".join(parts))
        sets = grad_sets(c)
        gcode, gnl, gnfl = gen_vrr("vrr", L + 1, sets, grad_sig=True)
        heavy = gnl > HEAVY_GRAD_VRR_LINES
        sizes = {s[0]: n_range(s[1], s[2]) * n_range(s[3], s[4]) for s in sets}
        gparts = [f"// Generated by gen_eri.py: gradient of class ({nm[:2]}|{nm[2:]}).\n#pragma once\n\n"]
        hr = grad_hrrs(c)
        gparts.append(f"struct GCls_{nm} {{\n  static constexpr int LA={la}, LB={lb}, LC={lc}, LD={ld}, L={L + 1}, "
                      f"HEAVY={int(heavy)}, HAS_U={int('accU' in sizes)}, "
                      + ", ".join(f"N_{k}={sizes.get(k, 1)}" for k in ["accU", "accA", "accB", "accC"])
                      + f", VRR_FLOPS={gnfl};\n")
        if not heavy:
            gparts.append(gcode)
            for hname, (a_, b_, c_, d_), src in hr:
                elo, ehi, flo, fhi = set_range(sets, src)
                h, _ = gen_hrr(f"hrr{hname}", a_, b_, c_, d_, elo, ehi, flo, fhi)
                gparts.append(h)
        gparts.append("};\n")
        write_if_changed(os.path.join(outdir, f"grad_{nm}.cuh"), "".join(gparts))
        if heavy:
            tape_all.append((nm, gen_tape(c)))
        stats.append((nm, nl, nfl, nh, gnl, gnfl, heavy))
    # tapes: one header per heavy class with the op arrays (host side; the
    # class's translation unit uploads them)
    for nm, (ops, accops, hops, nslot, accb, outs, nvrr) in tape_all:
        def arr(name, rows):
            flat = [str(x) for r in rows for x in r]
            lines = []
            for i in range(0, len(flat), 24):
                lines.append(", ".join(flat[i:i + 24]))
            return f"static const int {name}[] = {{\n" + ",\n".join(lines) + "\n};\n"
        tp = [f"// Generated by gen_eri.py: op tape of the gradient of class {nm}.\n"
              "// Op = 8 ints {kind, dst, s1, s2, s3, s4, s5, aux}; kind 0/1 bra/ket VRR,\n"
              "// 2 accumulate (aux = weight), 3/4 bra/ket HRR (aux = direction).\n#pragma once\n\n"]
        tp.append(arr("tape_vrr", ops))
        tp.append(arr("tape_acc", accops))
        tp.append(arr("tape_hrr", hops))
        for hname in HRR_NAMES:
            vals = outs.get(hname, [0])
            tp.append(f"static const int tape_out{hname}[] = {{" + ", ".join(map(str, vals)) + "};\n")
        tp.append(f"struct Tape_{nm} {{ static constexpr int NVRR={len(ops)}, NACC={len(accops)}, "
                  f"NHRR={len(hops)}, NSLOT={nslot}; }};\n")
        write_if_changed(os.path.join(outdir, f"grad_tape_{nm}.cuh"), "".join(tp))
    return stats


if __name__ == "__main__":
    st = generate(sys.argv[1] if len(sys.argv) > 1 else "gen")
    for s in st:
        print(*s)
