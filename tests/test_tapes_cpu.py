"""Host-side checks of the generated cooperative tapes (no GPU): the
shared-memory slots of the recursion's intermediates are reassigned by
liveness, and a tape must compute the same accumulators and HRR outputs with
the compacted slots as with one slot per intermediate, whatever order the
ops of a level run in (the lanes of a warp take them in any order); the ops
of a level must be independent and the packed accumulation ops must decode
to what was packed."""
import os
import random
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                "paper_1601_02713_gb300", "csrc"))
import gen_eri as g  # noqa: E402


def _tape(c, grad, compact):
    if compact:
        return g.gen_coop(c, grad)
    orig = g._compact_slots
    g._compact_slots = lambda ops, lv, keep, lo: (ops, {}, max([lo] + [op[1] + 1 for op in ops]))
    try:
        return g.gen_coop(c, grad)
    finally:
        g._compact_slots = orig


def _run(t, seed):
    """Interpret a tape as the kernels do (encoded words, level by level, the
    ops of a level in a shuffled order) for three primitive quartets."""
    rng = np.random.default_rng(seed)
    shuf = random.Random(seed)
    F0, L = t["F0"], t["L"]
    sm = np.full(F0 + t["nwork"] + 1, np.nan)
    sm[:t["nacc"]] = 0.0
    words = [[x & 0xffffffff for x in w] for w in g.encode_vrr_levels(t["vrr"], t["vrr_lv"])]
    acc = [g.encode_acc(op) & 0xffffffff for op in t["acc"]]
    lv = t["vrr_lv"]
    for _ in range(3):
        ct = rng.uniform(0.5, 1.5, 64)
        sm[F0:F0 + L + 1] = rng.uniform(0.5, 1.5, L + 1)
        for a in range(len(lv) - 1):
            idx = list(range(lv[a], lv[a + 1]))
            shuf.shuffle(idx)
            for o in idx:
                w0, w1, w2, w3 = words[o]
                n = w3 >> 30
                terms = [(w3 & 63, w0 >> 16), ((w3 >> 6) & 63, w1 & 0xffff), ((w3 >> 12) & 63, w1 >> 16),
                         ((w3 >> 18) & 63, w2 & 0xffff), ((w3 >> 24) & 63, w2 >> 16)][:n + 2]
                sm[w0 & 0xffff] = sum(ct[c] * sm[s] for c, s in terms)
        wts = rng.uniform(0.5, 1.5, 4)
        wts[0] = 1.0
        idx = list(range(len(acc)))
        shuf.shuffle(idx)
        for o in idx:
            a = acc[o]
            sm[a & 0x3fff] += wts[a >> 28] * sm[(a >> 14) & 0x3fff]
    accs = sm[:t["nacc"]].copy()
    hc = rng.uniform(-1, 1, 6)
    outs = []
    for _, sops, slv, out in t["hrrs"]:
        for a in range(len(slv) - 1):
            idx = list(range(slv[a], slv[a + 1]))
            shuf.shuffle(idx)
            for o in idx:
                e0, e1 = (x & 0xffffffff for x in g.encode_hrr(sops[o]))
                sm[e0 & 0xffff] = sm[e0 >> 16] + hc[e1 >> 16] * sm[e1 & 0xffff]
        outs.append(np.array([sm[o] for o in out]))
    return accs, outs


@pytest.mark.parametrize("cls,grad", [((1, 1, 1, 1), True), ((2, 1, 2, 1), True), ((2, 2, 2, 1), True),
                                      ((2, 2, 2, 2), False), ((2, 1, 1, 0), False)])
def test_compacted_tape_computes_the_same(cls, grad):
    t0, t1 = _tape(cls, grad, False), _tape(cls, grad, True)
    assert t1["nwork"] <= t0["nwork"]
    a0, o0 = _run(t0, 7)
    a1, o1 = _run(t1, 7)
    assert np.all(np.isfinite(a1)) and all(np.all(np.isfinite(x)) for x in o1)
    np.testing.assert_allclose(a1, a0, rtol=1e-13, atol=0)
    for x, y in zip(o1, o0):
        np.testing.assert_allclose(x, y, rtol=1e-13, atol=0)


def test_levels_are_independent_and_ops_decode():
    for c in g.classes():
        if sum(c) < 4:
            continue
        for grad in (False, True):
            t = g.gen_coop(c, grad)
            lv = t["vrr_lv"]
            for a in range(len(lv) - 1):
                ops = t["vrr"][lv[a]:lv[a + 1]]
                dst = {op[1] for op in ops}
                assert len(dst) == len(ops)
                assert not any(x in dst for op in ops for x in op[2:7] if x >= 0)
            for _, sops, slv, _ in t["hrrs"]:
                for a in range(len(slv) - 1):
                    ops = sops[slv[a]:slv[a + 1]]
                    dst = {op[1] for op in ops}
                    assert len(dst) == len(ops)
                    assert not any(x in dst for op in ops for x in op[2:4] if x >= 0)
            dsts = [op[0] for op in t["acc"]]
            assert len(set(dsts)) == len(dsts)
            for op in t["acc"]:
                a = g.encode_acc(op) & 0xffffffff
                assert (a & 0x3fff, (a >> 14) & 0x3fff, a >> 28) == tuple(op[:3])
