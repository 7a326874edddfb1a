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
import heapq
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
    """Demand-driven [e0|f0]^(m) generator. Nodes are kept structured so that
    each recursion step can be emitted as one chain of fused multiply-adds
    with the integer factors folded into pre-scaled constants."""

    def __init__(self):
        self.memo = {}
        self.nodes = []      # (name, kind, i, t1, t2, k1, t3, t4, k2, t5)
        self.uses = {}
        self.n = 0

    def _use(self, t):
        if t is not None:
            self.uses[t] = self.uses.get(t, 0) + 1

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
        t3 = t4 = t5 = None
        k1 = k2 = 0
        if sum(f) > 0:
            kind = "ket"
            i = pick_dir(f)
            f1 = sub(f, i)
            t1, t2 = self.get(e, f1, m), self.get(e, f1, m + 1)
            if f1[i] > 0:
                f2 = sub(f1, i)
                t3, t4, k1 = self.get(e, f2, m), self.get(e, f2, m + 1), f1[i]
            if e[i] > 0:
                t5, k2 = self.get(sub(e, i), f1, m + 1), e[i]
        else:
            kind = "bra"
            i = pick_dir(e)
            e1 = sub(e, i)
            t1, t2 = self.get(e1, f, m), self.get(e1, f, m + 1)
            if e1[i] > 0:
                e2 = sub(e1, i)
                t3, t4, k1 = self.get(e2, f, m), self.get(e2, f, m + 1), e1[i]
        for t in (t1, t2, t3, t4, t5):
            self._use(t)
        name = f"v{self.n}"
        self.n += 1
        self.nodes.append((name, kind, i, t1, t2, k1, t3, t4, k2, t5))
        self.memo[key] = name
        return name

    @staticmethod
    def const(base, k, used):
        if k == 1:
            return base
        used.add((base, k))
        return f"{base}_{k}"

    def expr(self, node, addend, used):
        """FMA chain of one recursion step; `addend` (or None) is added last.
        Returns (expression, flop count)."""
        name, kind, i, t1, t2, k1, t3, t4, k2, t5 = node
        if kind == "bra":
            a1, a2, c1, c2 = f"PA{i}", f"WP{i}", "o2p", "o2pr"
        else:
            a1, a2, c1, c2 = f"QC{i}", f"WQ{i}", "o2q", "o2qr"
        inner = addend
        fl = 0
        if t5 is not None:
            c = self.const("o2pq", k2, used)
            inner = f"fma({c}, {t5}, {inner})" if inner else f"{c}*{t5}"
            fl += 2 if addend or inner.startswith("fma") else 1
        if t3 is not None:
            ca, cb = self.const(c1, k1, used), self.const(c2, k1, used)
            inner = f"fma(-{cb}, {t4}, {inner})" if inner else f"-({cb}*{t4})"
            inner = f"fma({ca}, {t3}, {inner})"
            fl += 4
        inner = f"fma({a2}, {t2}, {inner})" if inner else f"{a2}*{t2}"
        fl += 2
        return f"fma({a1}, {t1}, {inner})", fl + 2


def level_range(lo, hi):
    out = []
    for l in range(max(lo, 0), hi + 1):
        out += carts(l)
    return out


def gen_vrr(name, Ltot, acc_sets, grad_sig=False):
    """acc_sets: list of (acc_name, e_lo, e_hi, f_lo, f_hi, weight_expr or None).
    Emits a device function adding [e0|f0]^(0) for every listed (e, f) into
    acc_name[idx] (times weight). A target that no other step reads and that
    is accumulated once without weight is accumulated inside its own FMA chain."""
    g = VRRGen()
    targets = []
    for acc, elo, ehi, flo, fhi, w in acc_sets:
        es = level_range(elo, ehi)
        fs = level_range(flo, fhi)
        for ie, e in enumerate(es):
            for jf, f in enumerate(fs):
                targets.append((acc, ie * len(fs) + jf, w, g.get(e, f, 0)))
    tcount = {}
    for _, _, _, v in targets:
        tcount[v] = tcount.get(v, 0) + 1
    fold = {}
    for acc, idx, w, v in targets:
        if w is None and tcount[v] == 1 and g.uses.get(v, 0) == 0 and v.startswith("v"):
            fold[v] = f"{acc}[{idx}]"
    used = set()
    lines = []
    nflop = 0
    for node in g.nodes:
        nm = node[0]
        if nm in fold:
            ex, fl = g.expr(node, fold[nm], used)
            lines.append(f"{fold[nm]} = {ex};")
        else:
            ex, fl = g.expr(node, None, used)
            lines.append(f"const R {nm} = {ex};")
        nflop += fl
    body_acc = []
    for acc, idx, w, v in targets:
        if v in fold:
            continue
        body_acc.append(f"{acc}[{idx}] = fma({w}, {v}, {acc}[{idx}]);" if w else f"{acc}[{idx}] += {v};")
        nflop += 2 if w else 1
    if grad_sig:
        args = "R* __restrict__ accU, R* __restrict__ accA, R* __restrict__ accB, R* __restrict__ accC, R wa, R wb, R wc"
    else:
        args = "R* __restrict__ acc"
    hdr = (f"template <typename R>\nstatic __device__ __forceinline__ void {name}(const R* __restrict__ Fm, "
           f"R PA0, R PA1, R PA2, R WP0, R WP1, R WP2, R QC0, R QC1, R QC2, R WQ0, R WQ1, R WQ2, "
           f"R o2p, R o2pr, R o2q, R o2qr, R o2pq, {args})\n{{\n")
    used_m = sorted({int(k[2]) for k in g.memo if sum(k[0]) == 0 and sum(k[1]) == 0})
    pre = "".join(f"    const R F{m} = Fm[{m}];\n" for m in used_m)
    pre += "".join(f"    const R {b}_{k} = R({k}) * {b};\n" for b, k in sorted(used))
    nflop += len(used)
    body = "\n".join("    " + l for l in lines + body_acc)
    return hdr + pre + body + "\n}\n", len(g.nodes), nflop


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


# ---------------------------------------------------------------------------
# Level-scheduled tapes for the cooperative kernels of the largest
# classes: every intermediate lives in shared memory and the ops of one
# dependency level are independent, so the 32 lanes of a warp execute a level
# in parallel, with a __syncwarp between levels. Slot layout: [0, NACC)
# accumulators, then F_m at F0 .. F0+L, then VRR intermediates; the HRR
# intermediates reuse the space from F0 on.
# Generator-side op = {kind, dst, s1, s2, s3, s4, s5, aux}: kind 0/1 bra/ket
# VRR (aux = dir | k1 << 4 | k2 << 8), kind 3/4 bra/ket HRR (aux = dir).
# Emitted forms (see coop_kernels.cuh):
#   VRR op = 4 ints, one fused multiply-add chain sum_t ct[c_t] sm[s_t] over
#     2..5 terms, ct = the primitive quartet's coefficient table (COOP_CT
#     entries); the ops of a level are sorted by their number of terms;
#   HRR op = 2 ints {dst | s1 << 16, s2 | coef << 16}: sm[dst] = sm[s1] +
#     hc[coef] sm[s2], hc = (AB_x, AB_y, AB_z, CD_x, CD_y, CD_z);
#   accumulation op = 4 ints {dst, src, weight, 0}.
# ---------------------------------------------------------------------------
# coefficient table of one primitive quartet: PA, WP, QC, WQ (0..11), then
# k o2p, -k o2pr, k o2q, -k o2qr, k o2pq for k = 1..5 (12..36)
COOP_KMAX = 5
CT_PA, CT_WP, CT_QC, CT_WQ = 0, 3, 6, 9
CT_O2P, CT_O2PR, CT_O2Q, CT_O2QR, CT_O2PQ = 12, 17, 22, 27, 32
COOP_CT = 37


def _i32(x):
    return x - (1 << 32) if x >= (1 << 31) else x


def encode_vrr(op):
    """(nterms, 4-int word) of one VRR op as a chain of products."""
    kind, d, s1, s2, s3, s4, s5, aux = op
    i, k1, k2 = aux & 15, (aux >> 4) & 15, aux >> 8
    assert k1 <= COOP_KMAX and k2 <= COOP_KMAX and max(d, s1, s2, s3, s4, s5) < 65536
    if kind == 0:
        terms = [(CT_PA + i, s1), (CT_WP + i, s2)]
        if s3 >= 0:
            terms += [(CT_O2P + k1 - 1, s3), (CT_O2PR + k1 - 1, s4)]
    else:
        terms = [(CT_QC + i, s1), (CT_WQ + i, s2)]
        if s3 >= 0:
            terms += [(CT_O2Q + k1 - 1, s3), (CT_O2QR + k1 - 1, s4)]
        if s5 >= 0:
            terms += [(CT_O2PQ + k2 - 1, s5)]
    n = len(terms)
    cs = [t[0] for t in terms] + [0] * (5 - n)
    ss = [t[1] for t in terms] + [0] * (5 - n)
    w = (d | (ss[0] << 16), ss[1] | (ss[2] << 16), ss[3] | (ss[4] << 16),
         cs[0] | (cs[1] << 6) | (cs[2] << 12) | (cs[3] << 18) | (cs[4] << 24) | ((n - 2) << 30))
    return n, [_i32(x) for x in w]


def encode_vrr_levels(ops, lv):
    """Encoded ops, each level's ops sorted by term count (a warp's round of
    32 ops then mostly runs one chain length)."""
    out = []
    for a in range(len(lv) - 1):
        enc = sorted((encode_vrr(op) for op in ops[lv[a]:lv[a + 1]]), key=lambda t: t[0])
        out += [w for _, w in enc]
    return out


def encode_acc(op):
    """One accumulation op {dst | src << 14 | weight << 28}."""
    dst, src, w, _ = op
    assert max(dst, src) < (1 << 14) and 0 <= w < 4
    return dst | (src << 14) | (w << 28)


def encode_hrr(op):
    kind, d, s1, s2, _, _, _, i = op
    assert max(d, s1, s2) < 65536
    return [_i32(d | (s1 << 16)), s2 | ((i if kind == 3 else 3 + i) << 16)]


# a class gets a cooperative tape above these VRR sizes (lines); its
# straight-line kernel is generated up to the MAX sizes; where both exist the
# autotuner picks one per class. For the Fock build the cooperative kernel is
# kept for (dd|dd) alone: timed on a full build it looked faster for (dp|pp)
# and (dp|dp) too, but in the SCF, whose builds are mostly incremental, it
# made the whole Fock build 28% slower.
COOP_ENERGY_MIN_VRR = 2000
STRAIGHT_ENERGY_MAX_VRR = 2000
COOP_GRAD_MIN_VRR = 400


def _sort_levels(ops, base_level):
    """Stable sort of ops by dependency level; returns (ops, level offsets)."""
    lvl = dict(base_level)
    out = []
    for op in ops:
        srcs = [x for x in op[2:7] if x >= 0]
        lv = 1 + max((lvl.get(x, 0) for x in srcs), default=0)
        lvl[op[1]] = lv
        out.append((lv, op))
    out.sort(key=lambda t: t[0])
    offs = [0]
    cur = 1
    for i, (lv, _) in enumerate(out):
        while lv > cur:
            offs.append(i)
            cur += 1
    offs.append(len(out))
    return [o for _, o in out], offs


def _compact_slots(ops, lv, keep, lo):
    """Shared-memory slots of the work nodes (ids >= lo, written by the
    level-sorted ops) reassigned by liveness: a node's slot is released once
    the last level that reads it has passed (the levels are separated by a
    barrier), and a level's results take the lowest released slots. Nodes in
    keep stay live to the end (read after the tape). Returns (ops, id map,
    one past the highest slot)."""
    last = {}
    for a in range(len(lv) - 1):
        for op in ops[lv[a]:lv[a + 1]]:
            for x in op[2:7]:
                if x >= lo:
                    last[x] = a
    end = len(lv)
    for x in keep:
        if x >= lo:
            last[x] = end
    free, top, mp = [], lo, {}
    release = {}
    for a in range(len(lv) - 1):
        for x in release.pop(a, []):
            heapq.heappush(free, x)
        for op in ops[lv[a]:lv[a + 1]]:
            d = op[1]
            slot = heapq.heappop(free) if free else top
            if slot == top:
                top += 1
            mp[d] = slot
            # a node nobody reads is released after its own level
            release.setdefault(last.get(d, a) + 1, []).append(slot)
    out = []
    for op in ops:
        out.append((op[0], mp[op[1]]) + tuple(mp.get(x, x) if x >= lo else x for x in op[2:7]) + (op[7],))
    return out, mp, top


def gen_coop(c, grad):
    la, lb, lc, ld = c
    L = la + lb + lc + ld + (1 if grad else 0)
    sets = grad_sets(c) if grad else [("acc", la, la + lb, lc, lc + ld, None)]
    acc_base, nacc = {}, 0
    for name, elo, ehi, flo, fhi, w in sets:
        acc_base[name] = nacc
        nacc += n_range(elo, ehi) * n_range(flo, fhi)
    F0 = nacc
    nxt = [F0 + L + 1]
    ops, memo = [], {}

    def new():
        v = nxt[0]
        nxt[0] += 1
        return v

    def get(e, f, m):
        if min(e) < 0 or min(f) < 0:
            return -1
        key = (e, f, m)
        if key in memo:
            return memo[key]
        if sum(e) == 0 and sum(f) == 0:
            memo[key] = F0 + m
            return F0 + m
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
            s5, k2 = -1, 0
            if e[i] > 0:
                s5, k2 = get(sub(e, i), f1, m + 1), e[i]
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

    wsel = {None: 0, "wa": 1, "wb": 2, "wc": 3}
    accops = []
    for name, elo, ehi, flo, fhi, w in sets:
        es, fs = level_range(elo, ehi), level_range(flo, fhi)
        for ie, e in enumerate(es):
            for jf, f in enumerate(fs):
                accops.append((acc_base[name] + ie * len(fs) + jf, get(e, f, 0), wsel[w], 0))
    vrr_ops, vrr_lv = _sort_levels(ops, {F0 + m: 0 for m in range(L + 1)})
    vrr_ops, vmap, vtop = _compact_slots(vrr_ops, vrr_lv, {a[1] for a in accops}, F0 + L + 1)
    accops = [(a[0], vmap.get(a[1], a[1]), a[2], a[3]) for a in accops]
    nwork = vtop - F0
    # HRR tapes: the class itself (energy) or the six shifted classes (gradient)
    targets = grad_hrrs(c) if grad else [("E", c, "acc")]
    hrrs = []
    for hname, (a_, b_, c_, d_), src in targets:
        elo, ehi, flo, fhi = set_range(sets, src)
        es, fs = level_range(elo, ehi), level_range(flo, fhi)
        eidx = {e: i for i, e in enumerate(es)}
        fidx = {f: i for i, f in enumerate(fs)}
        hm, hops = {}, []
        hn = [F0]

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
                kind = 4
            else:
                i = pick_dir(b)
                b1 = sub(b, i)
                s1, s2 = hget(add(a, i), b1, cc, dd), hget(a, b1, cc, dd)
                kind = 3
            dst = hn[0]
            hn[0] += 1
            hops.append((kind, dst, s1, s2, -1, -1, -1, i))
            hm[key] = dst
            return dst

        outs = [hget(a, b, cc, dd) for a in carts(a_) for b in carts(b_) for cc in carts(c_) for dd in carts(d_)]
        sops, slv = _sort_levels(hops, {})
        sops, hmap, htop = _compact_slots(sops, slv, set(outs), F0)
        outs = [hmap.get(o, o) if o >= F0 else o for o in outs]
        hrrs.append((hname, sops, slv, outs))
        nwork = max(nwork, htop - F0)
    return dict(L=L, nacc=nacc, F0=F0, nwork=nwork, vrr=vrr_ops, vrr_lv=vrr_lv, acc=accops, hrrs=hrrs)


def coop_header(nm, grad, t):
    """C++ header with the tape arrays of one class (host data, uploaded by
    the class's translation unit)."""
    pre = f"coop{'g' if grad else 'e'}_{nm}"

    def arr(name, flat):
        flat = [str(x) for x in flat]
        lines = [", ".join(flat[i:i + 24]) for i in range(0, len(flat), 24)] or ["0"]
        return f"static const int {name}[] = {{\n" + ",\n".join(lines) + "\n};\n"

    out = [f"// Generated by gen_eri.py: level-scheduled {'gradient' if grad else 'Fock'} tape of class {nm}.\n",
           "#pragma once\n\n"]
    out.append(arr(f"{pre}_vrr", [x for w in encode_vrr_levels(t["vrr"], t["vrr_lv"]) for x in w]))
    out.append(arr(f"{pre}_vrr_lv", t["vrr_lv"]))
    out.append(arr(f"{pre}_acc", [encode_acc(op) for op in t["acc"]]))
    names = []
    for hname, sops, slv, outs in t["hrrs"]:
        out.append(arr(f"{pre}_hrr{hname}", [x for op in sops for x in encode_hrr(op)]))
        out.append(arr(f"{pre}_hrr{hname}_lv", slv))
        out.append(arr(f"{pre}_out{hname}", outs))
        names.append((hname, len(sops), len(slv) - 1, len(outs)))
    out.append(f"struct Coop{'G' if grad else 'E'}_{nm} {{ static constexpr int L={t['L']}, NACC={t['nacc']}, "
               f"F0={t['F0']}, NWORK={t['nwork']}, NVRR={len(t['vrr'])}, NVLEV={len(t['vrr_lv']) - 1}, "
               f"NACCOP={len(t['acc'])}; }};\n")
    return "".join(out), names


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
        coop_e = nl > COOP_ENERGY_MIN_VRR
        straight_e = nl <= STRAIGHT_ENERGY_MAX_VRR
        if coop_e:
            hdr, _ = coop_header(nm, False, gen_coop(c, False))
            write_if_changed(os.path.join(outdir, f"coope_{nm}.cuh"), hdr)
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
        coop_g = gnl > COOP_GRAD_MIN_VRR
        if coop_g:
            hdr, _ = coop_header(nm, True, gen_coop(c, True))
            write_if_changed(os.path.join(outdir, f"coopg_{nm}.cuh"), hdr)
        stats.append((nm, nl, nfl, nh, gnl, gnfl, heavy, coop_e, coop_g, straight_e))
    return stats


if __name__ == "__main__":
    st = generate(sys.argv[1] if len(sys.argv) > 1 else "gen")
    for s in st:
        print(*s)
