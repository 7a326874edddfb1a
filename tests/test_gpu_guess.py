"""Learned initial density on the GPU against its oracle (oracle/guess.py) and
against the SCF itself.

* pair rows: the frame and the invariant features of every atom pair match
  the oracle's definitions (frames to FP64 round-off, features to FP32);
* block rotations: lab -> local and local -> lab blocks match M_A^T D M_B and
  M_A L M_B^T built from the oracle's shell representations;
* network: loss and gradients of the BF16 tensor-core network match FP64
  backpropagation run on the same BF16-rounded weights and inputs (relative
  error 1e-2 for the loss, 3e-2 in norm per parameter tensor: the
  activations and output gradients are rounded to BF16 before each GEMM);
* training lowers the loss; the learned guess converges to the same energy
  and gradient as the core-Hamiltonian guess (and, on a water dimer, as the
  oracle) in fewer SCF iterations on held-out geometries.
"""
import numpy as np
import pytest

import oracle as O
from oracle import guess as OG
from paper_1601_02713_gb300 import inputs, native

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

E_TOL = 1e-8
G_TOL = 1e-6


def _nsph(l):
    return 2 * l + 1


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return native.Context(0)


@pytest.fixture(scope="module")
def spd():
    bas = inputs.basis_set("split_spd")
    return bas, native.Basis(bas)


@pytest.fixture(scope="module")
def model(ctx, spd):
    return native.GuessModel(spd[1], seed=7)


def _shell_ls(bas):
    return {Z: [sh.l for sh in shells] for Z, shells in bas.items()}


def _atom_offsets(bas, Z):
    ls = _shell_ls(bas)
    off, n = [], 0
    for z in Z:
        off.append(n)
        n += sum(_nsph(l) for l in ls[int(z)])
    return off, n


def _geometries():
    r, _ = inputs.workload("water8_spd_32beads", nrep=1)
    Z, X = r.stacked()
    yield "water8", Z, X[0]
    Zh, Xh = inputs.small_molecule("h2")
    yield "h2", Zh, Xh
    # linear O-H-H: the reference atom of the O-H pair lies on the pair axis
    yield "linear", np.array([8, 1, 1], np.int32), np.array([[0.0, 0, 0], [0, 0, 1.8], [0, 0, 3.6]])
    Zw, Xw = inputs.small_molecule("water")
    yield "water", Zw, Xw


@pytest.mark.parametrize("case", [g[0] for g in _geometries()])
def test_pair_frames_and_features(model, case):
    _, Z, xyz = next(g for g in _geometries() if g[0] == case)
    out = model.pair_data(Z, xyz)
    n = len(Z)
    assert len(out["pairs"]) == n * (n + 1) // 2
    seen = set()
    elem_rank = {1: 0, 6: 1, 8: 2}
    for i, (A, B) in enumerate(out["pairs"]):
        assert elem_rank[int(Z[A])] >= elem_rank[int(Z[B])]
        seen.add((min(A, B), max(A, B)))
        np.testing.assert_allclose(out["frames"][i], OG.pair_frame(xyz, A, B), atol=1e-12, err_msg=f"{A},{B}")
        f = OG.pair_features(Z, xyz, A, B)
        np.testing.assert_allclose(out["feats"][i], f, rtol=2e-7, atol=1e-6, err_msg=f"{A},{B}")
    assert len(seen) == n * (n + 1) // 2


def test_block_rotations(model, spd):
    bas, _ = spd
    r, _ = inputs.workload("water8_spd_32beads", nrep=2)
    Z, X = r.stacked()
    xyz = X[1]
    off, N = _atom_offsets(bas, Z)
    ls = _shell_ls(bas)
    nb = {z: sum(_nsph(l) for l in ls[z]) for z in ls}
    rng = np.random.default_rng(3)
    D = rng.normal(size=(N, N)) * 0.2
    D = D + D.T
    nout = sum(nb[int(Z[A])] * nb[int(Z[B])] for A in range(len(Z)) for B in range(A, len(Z)))
    L = (rng.normal(size=nout) * 0.3).astype(np.float32)
    out = model.pair_data(Z, xyz, D=D, local_in=L, nbf=N)
    Dref = np.zeros((N, N))
    ncut = 0
    for i, (A, B) in enumerate(out["pairs"]):
        U = OG.pair_frame(xyz, A, B)
        MA = OG.atom_rotation(ls[int(Z[A])], U)
        MB = OG.atom_rotation(ls[int(Z[B])], U)
        na, nbB = MA.shape[0], MB.shape[0]
        o = out["block_off"][i]
        blk = D[off[A]:off[A] + na, off[B]:off[B] + nbB]
        ref = OG.to_local(blk, MA, MB)
        got = out["local"][o:o + na * nbB].reshape(na, nbB)
        np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6)
        if np.linalg.norm(xyz[A] - xyz[B]) <= OG.RCUT:
            Lb = L[o:o + na * nbB].reshape(na, nbB).astype(np.float64)
            if A == B:
                Lb = 0.5 * (Lb + Lb.T)
            lab = OG.to_lab(Lb, MA, MB)
            Dref[off[A]:off[A] + na, off[B]:off[B] + nbB] = lab
            Dref[off[B]:off[B] + nbB, off[A]:off[A] + na] = lab.T
        else:
            ncut += 1
    assert ncut > 0
    np.testing.assert_allclose(out["D_lab"], Dref, atol=1e-12)


def _bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _split_params(P, widths):
    """Layers of the flat parameter vector: 3 hidden (96->256, 256->256 x2),
    then one head per type (256 -> widths[t])."""
    layers = []
    o = 0
    dims = [(96, 256), (256, 256), (256, 256)] + [(256, w) for w in widths]
    for fi, fo in dims:
        W = P[o:o + fi * fo].reshape(fi, fo)
        o += fi * fo
        b = P[o:o + fo]
        o += fo
        layers.append((W, b))
    assert o == len(P)
    return layers


@pytest.mark.parametrize("ptype", [2, 5])
def test_mlp_gradients_against_fp64_backprop(model, spd, ptype):
    bas, _ = spd
    ls = _shell_ls(bas)
    nb = {e: sum(_nsph(l) for l in ls[z]) for e, z in enumerate((1, 6, 8))}
    pairs = [(0, 0), (1, 1), (2, 2), (2, 2), (2, 1), (2, 0), (1, 1), (1, 0), (0, 0)]
    widths = [nb[a] * nb[b] for a, b in pairs]
    # realistic inputs: features of the water8 pairs
    r, _ = inputs.workload("water8_spd_32beads", nrep=1)
    Z, X = r.stacked()
    feats = model.pair_data(Z, X[0])["feats"]
    rng = np.random.default_rng(11)
    n = 260
    Xin = feats[rng.integers(0, len(feats), n)]
    Y = (rng.normal(size=(n, widths[ptype])) * 0.2).astype(np.float32)
    loss, P, G = model.mlp_grad(ptype, Xin, Y)
    layers = _split_params(P.astype(np.float64), widths)
    params = [(_bf16(W), b) for W, b in layers[:3]] + [(_bf16(layers[3 + ptype][0]), layers[3 + ptype][1])]
    Lref, gref = OG.mse_loss_and_grads(params, _bf16(Xin), Y.astype(np.float64))
    assert abs(loss - Lref) / Lref < 1e-2, (loss, Lref)
    glayers = _split_params(G.astype(np.float64), widths)
    got = glayers[:3] + [glayers[3 + ptype]]
    for k, ((gW, gb), (rW, rb)) in enumerate(zip(got, gref)):
        eW = np.linalg.norm(gW - rW) / np.linalg.norm(rW)
        eb = np.linalg.norm(gb - rb) / np.linalg.norm(rb)
        assert eW < 3e-2 and eb < 3e-2, (k, eW, eb)
    for t in range(9):
        if t != ptype:
            assert not np.any(glayers[3 + t][0]) and not np.any(glayers[3 + t][1])


# ------------------------------------------------------------------ training and use
@pytest.fixture(scope="module")
def trained(ctx, spd):
    bas, B = spd
    m = native.GuessModel(B, seed=1)
    for reps in inputs.water_cluster_set(4, 6, 8, 50):
        Z, X = reps.stacked()
        info = m.add_data(ctx, B, Z, X)
        assert all(i["converged"] for i in info)
    assert m.ndata == 48
    hist = m.train(300, lr=1e-3)
    return m, hist


def test_training_lowers_the_loss(trained):
    m, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.1 * hist[0], (hist[0], hist[-1])
    assert abs(m.loss() - hist[-1]) < 0.5 * hist[-1]


def test_learned_guess_same_answer_fewer_iterations(ctx, spd, trained):
    bas, B = spd
    m, _ = trained
    held = inputs.water_cluster_set(4, 1, 6, 90)[0]
    Z, X = held.stacked()
    ctx.clear_guess()
    E0, G0, i0, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=0))
    m.attach(ctx)
    E1, G1, i1, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=2))
    assert all(i["converged"] for i in i0 + i1)
    np.testing.assert_allclose(E1, E0, atol=E_TOL, rtol=0)
    np.testing.assert_allclose(G1, G0, atol=G_TOL, rtol=0)
    it0 = np.array([i["iterations"] for i in i0])
    it1 = np.array([i["iterations"] for i in i1])
    assert it1.mean() < it0.mean(), (it0, it1)


def test_learned_guess_beats_sad_on_held_out_geometries(ctx, spd, trained):
    """Where no previous MOs exist (a first step, a new image), the learned
    density is the starting point to beat the superposition of atomic
    densities: on 18 beads of three held-out (H2O)4 geometry sets it takes
    fewer SCF iterations than SAD on average, and reaches the same answer."""
    bas, B = spd
    m, _ = trained
    m.attach(ctx)
    its = {4: [], 2: []}
    for seed in (90, 91, 92):
        held = inputs.water_cluster_set(4, 1, 6, seed)[0]
        Z, X = held.stacked()
        out = {}
        for g in (4, 2):
            ctx.clear_guess()
            E, G, info, rc = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=g))
            assert rc == 0 and all(i["converged"] for i in info)
            its[g] += [i["iterations"] for i in info]
            out[g] = (E, G)
        np.testing.assert_allclose(out[2][0], out[4][0], atol=E_TOL, rtol=0)
        np.testing.assert_allclose(out[2][1], out[4][1], atol=G_TOL, rtol=0)
    assert np.mean(its[2]) < np.mean(its[4]), (its[4], its[2])


def test_learned_guess_against_oracle(ctx, spd, trained):
    bas, B = spd
    m, _ = trained
    r, _ = inputs.workload("water2_min_4beads", nrep=1)
    Z, X = r.stacked()
    m.attach(ctx)
    E, G, info, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=2))
    assert info[0]["converged"]
    E0, G0, _ = O.rhf_energy_gradient(bas, Z, X[0])
    assert abs(E[0] - E0) < E_TOL
    np.testing.assert_allclose(G[0], G0, atol=G_TOL, rtol=0)


def test_cache_then_learned_guess(ctx, spd, trained):
    """guess = 3: replicas without cached MOs start from the learned density,
    then from their own MOs."""
    bas, B = spd
    m, _ = trained
    held = inputs.water_cluster_set(4, 1, 3, 91)[0]
    Z, X = held.stacked()
    m.attach(ctx)
    ctx.clear_guess()
    E1, _, i1, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=3))
    E2, _, i2, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=3))
    np.testing.assert_allclose(E2, E1, atol=E_TOL, rtol=0)
    assert max(i["iterations"] for i in i2) <= 3


def test_save_load_roundtrip(ctx, spd, trained, tmp_path):
    bas, B = spd
    m, _ = trained
    p = tmp_path / "guess.bin"
    m.save(str(p))
    m2 = native.GuessModel(B, seed=99)
    m2.load_weights(str(p))
    held = inputs.water_cluster_set(4, 1, 2, 92)[0]
    Z, X = held.stacked()
    m.attach(ctx)
    E1, _, i1, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=2))
    m2.attach(ctx)
    E2, _, i2, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=2))
    assert [i["iterations"] for i in i1] == [i["iterations"] for i in i2]
    # the same start: equal to the round-off of the Fock build's atomic accumulation
    np.testing.assert_allclose(E1, E2, atol=1e-10, rtol=0)


def test_learned_guess_errors(ctx, spd):
    bas, B = spd
    Z, X = inputs.small_molecule("water")
    c2 = native.Context(0)
    with pytest.raises(native.PimdError) as e:
        native.pimd_bo_forces(c2, B, Z, X[None], native.scf_opts(guess=2))
    assert e.value.code == native.PIMD_EINVAL
    # a model of the minimal basis does not fit the split-valence basis
    mmin = native.GuessModel(native.Basis(inputs.basis_set("min_sp")), seed=0)
    mmin.attach(c2)
    with pytest.raises(native.PimdError) as e:
        native.pimd_bo_forces(c2, B, Z, X[None], native.scf_opts(guess=2))
    assert e.value.code == native.PIMD_EINVAL
    c2.close()


# ------------------------------------------------------------------ SAD guess
@pytest.mark.parametrize("kind,Z", [("split_spd", 8), ("split_spd", 6), ("split_spd", 1), ("min_sp", 8),
                                    ("min_sp", 1)])
def test_sad_atomic_density_against_oracle(ctx, kind, Z):
    bas = inputs.basis_set(kind)
    B = native.Basis(bas)
    D = native.pimd_sad_atomic_density(ctx, B, Z)
    np.testing.assert_allclose(D, O.sad_atomic_density(bas, Z), atol=1e-7)


def test_sad_guess_same_answer(ctx, spd):
    bas, B = spd
    r, _ = inputs.workload("water8_spd_32beads", nrep=2)
    Z, X = r.stacked()
    ctx.clear_guess()
    E0, G0, i0, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=0))
    E1, G1, i1, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=4))
    assert all(i["converged"] for i in i0 + i1)
    np.testing.assert_allclose(E1, E0, atol=E_TOL, rtol=0)
    np.testing.assert_allclose(G1, G0, atol=G_TOL, rtol=0)
    # guess = 5: the second call starts from the cached MOs
    ctx.clear_guess()
    native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=5))
    E2, _, i2, _ = native.pimd_bo_forces(ctx, B, Z, X, native.scf_opts(guess=5))
    np.testing.assert_allclose(E2, E0, atol=E_TOL, rtol=0)
    assert max(i["iterations"] for i in i2) <= 3


def test_sad_guess_ragged_images(ctx, spd):
    """C, H and O atoms; images of different sizes in one call."""
    bas, B = spd
    reps, _ = inputs.workload("da_images_24")
    sub = inputs.Replicas([reps.Z[i] for i in (0, 7)], [reps.coords[i] for i in (0, 7)])
    nat, Zc, Xc = sub.concat()
    E0, G0, i0, _ = native.string_images_forces(ctx, B, nat, Zc, Xc, native.scf_opts(guess=0))
    E1, G1, i1, _ = native.string_images_forces(ctx, B, nat, Zc, Xc, native.scf_opts(guess=4))
    assert all(i["converged"] for i in i0 + i1)
    np.testing.assert_allclose(E1, E0, atol=E_TOL, rtol=0)
    np.testing.assert_allclose(G1, G0, atol=G_TOL, rtol=0)
