"""GPU parity against the CPU oracle, through the C ABI.

Bars (the tolerances of the FP64 path): energies within 1e-8 hartree,
gradients within 1e-6 hartree/bohr of the oracle; intermediate quantities
(Boys values, one-electron matrices, Fock matrices of a fixed density) within
the round-off of FP64 sums of their size.
"""
import numpy as np
import pytest

import oracle as O
from paper_1601_02713_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

E_TOL = 1e-8
G_TOL = 1e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


@pytest.fixture(scope="module")
def spd():
    bas = inputs.basis_set("split_spd")
    return bas, native.Basis(bas)


def test_boys_function(ctx):
    rng = np.random.default_rng(0)
    T = np.concatenate([np.linspace(0, 45, 721), rng.uniform(0, 60, 2000), [1e-12, 39.999, 40.0, 40.001, 150.0]])
    Tt = torch.tensor(T, dtype=torch.float64, device="cuda")
    for m in [0, 1, 2, 5, 9, 12]:
        F = torch.empty_like(Tt)
        native.pimd_boys_dev(ctx, Tt, m, F)
        got = F.cpu().numpy()
        ref = np.array([O.boys(m, t) for t in T])
        rel = np.abs(got - ref) / ref
        assert rel.max() < 5e-14, (m, rel.max(), T[rel.argmax()])


# FP32 Boys evaluation of the mixed-precision quartets: largest relative
# error against the oracle (both branches: 4-term Taylor table below T = 40,
# asymptotic form with upward recursion above, e^-T dropped from T = 72 on)
BOYS_F32_REL = 1e-6


@pytest.mark.parametrize("variant", [0, 1])
def test_boys_function_fp32(ctx, variant):
    """The FP32 form of F_m(T), m = 0..12, against the oracle on a dense
    grid that straddles both switch points (T = 40: table -> asymptotic
    branch; T = 72: e^-T dropped) and on random T up to 100. Both branches
    stay within FP32 rounding of the recursion at the switches (the bound is
    stated per order in BOYS_F32_REL), so no FP64 fallback is needed there."""
    rng = np.random.default_rng(1)
    T = np.concatenate([np.arange(38.5, 41.5, 0.002), np.arange(70.5, 73.5, 0.002), rng.uniform(0, 100, 3000),
                        np.linspace(0, 2, 200)]).astype(np.float32)
    Tt = torch.tensor(T, dtype=torch.float32, device="cuda")
    Td = T.astype(np.float64)   # the reference at the float argument itself
    for m in range(13):
        F = torch.empty_like(Tt)
        native.pimd_boys_f32_dev(ctx, Tt, m, F, variant)
        got = F.cpu().numpy().astype(np.float64)
        ref = np.array([O.boys(m, t) for t in Td])
        rel = np.abs(got - ref) / ref
        assert rel.max() < BOYS_F32_REL, (variant, m, rel.max(), Td[rel.argmax()])
        near = np.abs(Td - 40.0) < 1.0
        assert rel[near].max() < BOYS_F32_REL, (variant, m, "T near 40", rel[near].max())


@pytest.mark.parametrize("mol", ["water", "dimer"])
def test_one_electron_matrices(ctx, spd, mol):
    bas, B = spd
    if mol == "water":
        Z, X = inputs.small_molecule("water")
    else:
        r, _ = inputs.workload("water2_min_4beads")
        Z, Xs = r.stacked()
        X = Xs[1]
    S, T, V = native.pimd_one_electron(ctx, B, Z, X)
    ob = O.OracleBasis.build(bas, Z, X)
    S0, T0, V0 = O.one_electron(ob, Z, X)
    np.testing.assert_allclose(S, S0, atol=1e-13)
    np.testing.assert_allclose(T, T0, atol=1e-11)
    np.testing.assert_allclose(V, V0, atol=1e-11)


def _random_density(N, nrep, seed):
    rng = np.random.default_rng(seed)
    D = rng.normal(size=(nrep, N, N)) * 0.3
    return D + D.transpose(0, 2, 1)


@pytest.mark.parametrize("mol,nrep", [("water", 1), ("water2_spd", 3)])
def test_fock_matrix_of_fixed_density(ctx, spd, mol, nrep):
    bas, B = spd
    if mol == "water":
        Z, X = inputs.small_molecule("water")
        Xs = np.stack([X] * nrep)
    else:
        r, _ = inputs.workload("water2_min_4beads", nrep=nrep)
        Z, Xs = r.stacked()
    N = B.nbf(Z)
    D = _random_density(N, nrep, 7)
    Dt = torch.tensor(D, device="cuda")
    Gt = torch.zeros_like(Dt)
    native.pimd_fock_dev(ctx, B, Z, Xs, Dt, Gt, 1e-12)
    G = Gt.cpu().numpy()
    for k in range(nrep):
        ob = O.OracleBasis.build(bas, Z, Xs[k])
        J, K, _ = O.jk(ob, D[k], 1e-12)
        ref = J - 0.5 * K
        err = np.abs(G[k] - ref).max()
        assert err < 1e-10 * max(1.0, np.abs(ref).max()), (k, err)


def _oracle_eg(bas, Z, X):
    E, G, res = O.rhf_energy_gradient(bas, Z, X)
    assert res.converged
    return E, G


def test_water_dimer_min_basis_4_beads(ctx):
    reps, kind = inputs.workload("water2_min_4beads")
    Z, Xs = reps.stacked()
    bas = inputs.basis_set(kind)
    B = native.Basis(bas)
    E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, Xs)
    assert rc == 0
    for k in range(len(Xs)):
        E0, G0 = _oracle_eg(bas, Z, Xs[k])
        assert abs(E[k] - E0) < E_TOL, (k, E[k], E0)
        assert np.abs(G[k] - G0).max() < G_TOL, (k, np.abs(G[k] - G0).max())
        assert info[k]["converged"] == 1


def test_water_monomer_spd(ctx, spd):
    bas, B = spd
    Z, X = inputs.small_molecule("water")
    E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, X[None])
    assert rc == 0
    E0, G0 = _oracle_eg(bas, Z, X)
    assert abs(E[0] - E0) < E_TOL
    assert np.abs(G[0] - G0).max() < G_TOL
    assert np.abs(G[0].sum(0)).max() < 1e-9


def test_batched_equals_single(ctx, spd):
    bas, B = spd
    reps, _ = inputs.workload("water2_min_4beads", nrep=3)
    Z, Xs = reps.stacked()
    E, G, _, rc = native.pimd_bo_forces(ctx, B, Z, Xs)
    assert rc == 0
    for k in range(3):
        e1, g1, _, rc1 = native.pimd_bo_forces(ctx, B, Z, Xs[k:k + 1])
        assert rc1 == 0
        assert abs(e1[0] - E[k]) < 1e-11
        assert np.abs(g1[0] - G[k]).max() < 1e-10


def test_ragged_images(ctx, spd):
    bas, B = spd
    Zw, Xw = inputs.small_molecule("water")
    r, _ = inputs.workload("water2_min_4beads", nrep=2)
    Zd, Xd = r.stacked()
    mols = [(Zw, Xw), (Zd, Xd[0]), (Zw, Xw + 0.05), (Zd, Xd[1])]
    nat = [len(z) for z, _ in mols]
    Zc = np.concatenate([z for z, _ in mols])
    Xc = np.concatenate([x for _, x in mols])
    E, G, info, rc = native.string_images_forces(ctx, B, nat, Zc, Xc)
    assert rc == 0
    off = 0
    for k, (z, x) in enumerate(mols):
        E0, G0 = _oracle_eg(bas, z, x)
        assert abs(E[k] - E0) < E_TOL, (k, E[k] - E0)
        assert np.abs(G[off:off + len(z)] - G0).max() < G_TOL
        off += len(z)


def test_mo_reuse_guess_matches_core_guess(ctx):
    """Sec. 2: each replica's MOs are reused as the next step's guess; the
    converged result must not depend on the guess."""
    reps, kind = inputs.workload("water2_min_4beads")
    bas = inputs.basis_set(kind)
    B = native.Basis(bas)
    seq = inputs.markov_steps(reps, 3, seed=5)
    ctx.clear_guess()
    res = {}
    for gs in (1, 0):
        ctx.clear_guess()
        for s in range(3):
            Z, X = seq[s].stacked()
            E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=gs))
            assert rc == 0
            res[(gs, s)] = (E, G, [i["iterations"] for i in info])
    for s in range(3):
        E1, G1, it1 = res[(1, s)]
        E0, G0, it0 = res[(0, s)]
        assert np.abs(E1 - E0).max() < 1e-9
        assert np.abs(G1 - G0).max() < 1e-7
        if s > 0:
            assert np.mean(it1) <= np.mean(it0)


def test_mixed_precision_fp32_quartets(ctx, spd):
    """Quartets whose bound Q_ab Q_cd max|dD| is below 1e-6 run in FP32: the
    mixed path's bar is 1e-6 Eh and 1e-5 Eh/bohr against the oracle; it must
    actually route quartets to FP32 and stay close to the FP64 path."""
    bas, B = spd
    reps, _ = inputs.workload("water2_min_4beads", nrep=2)
    Z, Xs = reps.stacked()
    E64, G64, _, rc = native.pimd_bo_forces(ctx, B, Z, Xs)
    assert rc == 0
    E32, G32, info, rc = native.pimd_bo_forces(ctx, B, Z, Xs, native.scf_opts(fp32_tau=1e-6))
    assert rc == 0
    st = native.pimd_last_stats(ctx)
    assert st["quartets_fp32"] > 0
    # per-replica split of the executed quartets: every replica routes some
    # to FP32, and the records add up to the call's counters
    assert all(i["nq_fp32"] > 0 and i["nq_fp64"] > 0 for i in info)
    assert sum(i["nq_fp32"] for i in info) == st["quartets_fp32"]
    assert sum(i["nq_fp64"] for i in info) == st["quartets_fp64"]
    assert np.abs(E32 - E64).max() < 1e-7
    assert np.abs(G32 - G64).max() < 1e-6
    for k in range(len(Xs)):
        E0, G0 = _oracle_eg(bas, Z, Xs[k])
        assert abs(E32[k] - E0) < 1e-6
        assert np.abs(G32[k] - G0).max() < 1e-5


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    return json.load(open(path))


@pytest.mark.parametrize("fp32_tau", [0.0, 1e-6])
def test_water8_full_size_against_stored_oracle(ctx, spd, fp32_tau):
    """(H2O)8, 192 functions: the first bead of the benchmark workload, in the
    batched launch of 4 beads the benchmark uses, against the oracle's energy
    and gradient stored by tests/golden/make_golden.py."""
    bas, B = spd
    g = _golden("water8_spd_32beads_rep0.json")
    reps, _ = inputs.workload("water8_spd_32beads", nrep=4)
    Z, Xs = reps.stacked()
    assert np.abs(Xs[0] - np.array(g["coords_bohr"])).max() < 1e-12
    E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, Xs, native.scf_opts(fp32_tau=fp32_tau))
    assert rc == 0
    etol, gtol = (E_TOL, G_TOL) if fp32_tau == 0 else (1e-6, 1e-5)
    assert abs(E[0] - g["energy"]) < etol, E[0] - g["energy"]
    assert np.abs(G[0] - np.array(g["gradient"])).max() < gtol
    assert np.abs(G.sum(axis=1)).max() < 1e-8


@pytest.mark.parametrize("fp32_tau,tol", [(0.0, 1e-8), (1e-6, 1e-7)])
def test_water32_full_size_sampled_fock_blocks(ctx, spd, fp32_tau, tol):
    """(H2O)32, 768 functions (the largest workload): the full Fock-build
    launch for one bead with a seeded density of SCF-like magnitude, checked
    on sampled shell-pair blocks that the oracle computes from the definition
    (every ordered shell pair, no screening): s-s on one atom, p-s across the
    cluster, d-p and d-d blocks."""
    bas, B = spd
    reps, _ = inputs.workload("water32_spd_16beads", nrep=1)
    Z, Xs = reps.stacked()
    ob = O.OracleBasis.build(bas, Z, Xs[0])
    N = ob.nbf
    rng = np.random.default_rng(32)
    Cocc = rng.normal(size=(N, 160)) / np.sqrt(N)
    D = 2.0 * Cocc @ Cocc.T
    Dt = torch.tensor(D[None], device="cuda")
    Gt = torch.zeros_like(Dt)
    native.pimd_fock_dev(ctx, B, Z, Xs, Dt, Gt, 1e-12, fp32_tau)
    G = Gt[0].cpu().numpy()
    off = np.cumsum([0] + [ob.shell_nbf(s) for s in range(len(ob.l))])
    ls = np.asarray(ob.l)
    d_sh = np.nonzero(ls == 2)[0]
    p_sh = np.nonzero(ls == 1)[0]
    s_sh = np.nonzero(ls == 0)[0]
    picks = [(s_sh[0], s_sh[1]), (p_sh[3], s_sh[-5]), (d_sh[7], p_sh[40]), (d_sh[20], d_sh[21])]
    for a, b in picks:
        ref = O.g_block(ob, D, int(a), int(b))
        got = G[off[a]:off[a + 1], off[b]:off[b + 1]]
        err = np.abs(got - ref).max()
        assert err < tol * max(1.0, np.abs(ref).max()), (a, b, err)


def test_autotune_keeps_results(spd):
    """Tile widths picked by the autotuner change the work decomposition
    only: energies and gradients stay within round-off."""
    bas, B = spd
    c = native.Context(0)
    r, _ = inputs.workload("water8_spd_32beads", nrep=2)
    Z, X = r.stacked()
    E0, G0, _, _ = native.pimd_bo_forces(c, B, Z, X)
    widths, gvar, ms = native.pimd_autotune(c, B, Z, X)
    assert len(widths) == 21 and all(w in (0, 32, 64, 128) for w in widths) and ms > 0
    assert all(v in (0, 1) for v in gvar)
    c.clear_guess()
    E1, G1, info, _ = native.pimd_bo_forces(c, B, Z, X)
    assert all(i["converged"] for i in info)
    np.testing.assert_allclose(E1, E0, atol=1e-10, rtol=0)
    np.testing.assert_allclose(G1, G0, atol=1e-9, rtol=0)
    c.close()


def test_graph_replay_matches_plain_launches(ctx, spd):
    """use_graphs = 0 (plain launches) and 1 (CUDA graphs from the second SCF
    iteration on) give the same energies, gradients and iteration counts."""
    bas, B = spd
    r, _ = inputs.workload("water8_spd_32beads", nrep=3)
    Z, X = r.stacked()
    ctx.clear_guess()
    E0, G0, i0, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(use_graphs=0))
    ctx.clear_guess()
    E1, G1, i1, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(use_graphs=1))
    assert [i["iterations"] for i in i0] == [i["iterations"] for i in i1]
    np.testing.assert_allclose(E1, E0, atol=1e-10, rtol=0)
    np.testing.assert_allclose(G1, G0, atol=1e-9, rtol=0)


def test_scf_trace_and_fock_times_are_consistent(ctx, spd):
    """The per-iteration records of a call agree with its statistics and with
    the rules of the SCF loop: one trace row per iteration of each replica,
    the first build and the converging one full, the accepted step within
    the energy bar, one Fock record per iteration of the longest replica,
    their times summing to the call's Fock time and their quartets to the
    executed quartets; the last incremental build, whose density change is
    small, executes fewer quartets than the full first build (the early
    ones need not: the change of a start density can be as large as the
    density)."""
    bas, B = spd
    r, _ = inputs.workload("water8_spd_32beads", nrep=3)
    Z, X = r.stacked()
    ctx.clear_guess()
    E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts())
    assert rc == 0
    st = native.pimd_last_stats(ctx)
    for k, inf in enumerate(info):
        tr = native.pimd_last_trace(ctx, k)
        assert len(tr["energy"]) == inf["iterations"]
        assert tr["full_build"][0] == 1 and tr["full_build"][-1] == 1
        assert tr["energy"][-1] == pytest.approx(E[k], abs=1e-12)
        assert abs(tr["energy"][-1] - tr["energy"][-2]) < 1e-10
        assert tr["error"][-1] < 1e-8
    ft = native.pimd_last_fock_times(ctx)
    assert len(ft["ms"]) == max(i["iterations"] for i in info) == st["fock_builds"]
    assert np.all(ft["ms"] > 0)
    assert ft["ms"].sum() == pytest.approx(st["ms_fock"], rel=1e-6)
    assert ft["quartets"].sum() == st["quartets_fp64"] + st["quartets_fp32"]
    assert 0 < ft["quartets"][0] <= st["nquartets_total"]
    assert sum(i["nq_fp64"] for i in info) == st["quartets_fp64"] and all(i["nq_fp32"] == 0 for i in info)
    assert all(0 < i["nq_fp64"] <= i["iterations"] * i["nquartets"] for i in info)
    tr0 = native.pimd_last_trace(ctx, 0)
    inc = [k for k in range(1, len(tr0["full_build"])) if tr0["full_build"][k] == 0]
    assert inc and ft["quartets"][inc[-1]] < ft["quartets"][0]
    # the gradient's executed work: every quartet at most once, and a
    # recursion of at least one operation per primitive quartet
    assert 0 < st["grad_quartets"] <= st["nquartets_total"]
    assert st["grad_flops"] > st["grad_quartets"] and st["grad_flops32"] == 0


@pytest.mark.parametrize("fp32_tau", [0.0, 1e-6])
def test_diels_alder_images_against_stored_oracle(ctx, spd, fp32_tau):
    """String images of uneven size (config 4): the stored oracle images in
    one ragged batch with their neighbours (C, H and O; 200-296 functions),
    energies and gradients against the oracle's values stored by
    tests/golden/make_golden.py."""
    import glob
    import os
    bas, B = spd
    files = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden", "da_images_24_rep*.json")))
    if not files:
        pytest.skip("no stored Diels-Alder oracle images")
    reps, _ = inputs.workload("da_images_24")
    gold = [_golden(os.path.basename(f)) for f in files]
    idx = sorted({g["replica"] for g in gold} | {4, 9})
    sub = inputs.Replicas([reps.Z[i] for i in idx], [reps.coords[i] for i in idx])
    nat, Zc, Xc = sub.concat()
    E, G, info, rc = native.string_images_forces(ctx, B, nat, Zc, Xc, native.scf_opts(fp32_tau=fp32_tau))
    assert rc == 0 and all(i["converged"] for i in info)
    etol, gtol = (E_TOL, G_TOL) if fp32_tau == 0 else (1e-6, 1e-5)
    off = np.concatenate([[0], np.cumsum(nat)])
    for g in gold:
        k = idx.index(g["replica"])
        assert np.abs(Xc[off[k]:off[k + 1]] - np.array(g["coords_bohr"])).max() < 1e-12
        assert abs(E[k] - g["energy"]) < etol, (g["replica"], E[k] - g["energy"])
        assert np.abs(G[off[k]:off[k + 1]] - np.array(g["gradient"])).max() < gtol


def test_deterministic_mode_is_bitwise_reproducible(spd):
    """deterministic = 1: the Fock increments, V_nn and the gradient are summed
    as fixed-point integers, so repeated calls (fresh contexts, the same
    inputs) give bitwise-identical energies and gradients, within round-off
    of the FP64-atomic default."""
    bas, B = spd
    reps, _ = inputs.workload("water8_spd_32beads", nrep=3)
    Z, X = reps.stacked()
    out = []
    for _ in range(2):
        c = native.Context(0)
        E, G, info, rc = native.pimd_bo_forces(c, B, Z, X, native.scf_opts(deterministic=1))
        assert rc == 0 and all(i["converged"] for i in info)
        out.append((E, G))
        c.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    c = native.Context(0)
    E0, G0, _, rc = native.pimd_bo_forces(c, B, Z, X)
    c.close()
    assert rc == 0
    np.testing.assert_allclose(out[0][0], E0, atol=1e-9, rtol=0)
    np.testing.assert_allclose(out[0][1], G0, atol=1e-8, rtol=0)


def _water32(nrep=1):
    reps, _ = inputs.workload("water32_spd_16beads", nrep=nrep)
    return reps.stacked()


def test_water32_full_fock_build_against_oracle(ctx, spd):
    """(H2O)32, 768 functions: one whole Fock build of bead 0 for the
    oracle's core-Hamiltonian density, against the oracle's build stored by
    tests/golden/make_fock_golden.py (every element through G v for two
    seeded vectors, the diagonal, two full rows, v^T G v and tr(D G))."""
    import importlib.util
    import os
    g = _golden("water32_spd_16beads_rep0_fock.json")
    spec = importlib.util.spec_from_file_location(
        "make_fock_golden", os.path.join(os.path.dirname(__file__), "golden", "make_fock_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    bas, B = spd
    Z, Xs = _water32()
    assert np.abs(Xs[0] - np.array(g["coords_bohr"])).max() < 1e-12
    ob, D = mk.core_density(bas, Z, Xs[0])
    Dt = torch.tensor(D[None], device="cuda")
    Gt = torch.zeros_like(Dt)
    native.pimd_fock_dev(ctx, B, Z, Xs[:1], Dt, Gt, 1e-12, 0.0)
    G = Gt[0].cpu().numpy()
    scale = np.abs(np.array(g["diag"])).max()
    for v, ref in zip(mk.probe_vectors(ob.nbf), g["Gv"]):
        assert np.abs(G @ v - np.array(ref)).max() < 1e-8 * scale * np.sqrt(ob.nbf)
    assert np.abs(np.diag(G) - np.array(g["diag"])).max() < 1e-9 * scale
    for r, row in g["rows"].items():
        assert np.abs(G[int(r)] - np.array(row)).max() < 1e-9 * scale
    assert abs(np.sum(D * G) - g["tr_DG"]) < 1e-8 * abs(g["tr_DG"])


def test_water32_bead_invariance_and_mixed_precision(ctx, spd):
    """(H2O)32 on the GPU alone, properties that hold at any size, on one
    bead (768 functions, SAD start): the mixed-precision energy is invariant
    under a rigid motion of the bead and its gradient turns with it; the
    mixed energy and gradient stay within the mixed tolerances (1e-6 Eh,
    1e-5 Eh/bohr) of the FP64 path. Also the first SCF at this size (the
    Jacobi eigensolver at n = 768, convergence with incremental builds)."""
    bas, B = spd
    Z, Xs = _water32()
    X = Xs[:1]
    E32, G32, i32, rc = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=4, fp32_tau=1e-6))
    assert rc == 0 and i32[0]["converged"], i32
    ang = 0.61
    c, s = np.cos(ang), np.sin(ang)
    Rm = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]]) @ np.array([[1.0, 0.0, 0.0], [0.0, c, s],
                                                                          [0.0, -s, c]])
    Xr = X @ Rm.T + np.array([0.7, -1.1, 0.4])
    Er, Gr, ir, rc = native.pimd_bo_forces(ctx, B, Z, Xr, native.scf_opts(guess=4, fp32_tau=1e-6))
    assert rc == 0 and ir[0]["converged"], ir
    assert abs(Er[0] - E32[0]) < 1e-8
    assert np.abs(Gr[0] - G32[0] @ Rm.T).max() < 1e-6
    E64, G64, i64, rc = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=4))
    assert rc == 0 and i64[0]["converged"], i64
    assert abs(E32[0] - E64[0]) < 1e-6
    assert np.abs(G32 - G64).max() < 1e-5
