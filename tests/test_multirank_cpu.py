"""Replica parallelism on CPU ranks (gloo, world size 2): the step's
replicas are split into contiguous blocks (beads evenly, string images of
uneven size by their estimated cost), each rank evaluates its block, and one
all-gather gives every rank every replica's energy and gradient. The
gathered results must equal a single-rank evaluation of the same step. The
per-replica evaluation here is a CPU stand-in with the interface of the
forces call (a pair potential), since these ranks have no GPU; the
benchmark's multi-rank timing rules (max over ranks, whole-job throughput)
are checked as well."""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1601_02713_gb300 import replicas as RP  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def pair_forces(Z_list, coords_list):
    """Stand-in for the forces call: E = sum_{i<j} Z_i Z_j exp(-r_ij) per
    replica, gradients concatenated over the replicas' atoms."""
    Es, Gs = [], []
    for Z, X in zip(Z_list, coords_list):
        X = np.asarray(X, float)
        Zf = np.asarray(Z, float)
        d = X[:, None, :] - X[None, :, :]
        r = np.sqrt((d ** 2).sum(-1)) + np.eye(len(Z))
        w = np.outer(Zf, Zf) * np.exp(-r)
        np.fill_diagonal(w, 0.0)
        Es.append(0.5 * w.sum())
        Gs.append(-(w / r)[:, :, None].__mul__(d).sum(1))
    return np.array(Es), np.concatenate(Gs)


def _step_inputs():
    from paper_1601_02713_gb300 import inputs
    reps, _ = inputs.workload("water2_min_4beads", nrep=5)
    da, _ = inputs.workload("da_images_24")
    return reps, da


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    from paper_1601_02713_gb300 import replicas as rp
    beads, da = _step_inputs()
    out = {}
    # beads of one molecule: even contiguous blocks (5 beads over 2 ranks: 3 + 2)
    E, G, blocks = rp.distributed_step(pair_forces, beads.Z, beads.coords, rank, world, dist)
    out["beads"] = (E.numpy(), G.numpy(), blocks)
    # string images of uneven size, balanced by a cost per image
    costs = [len(z) ** 4 for z in da.Z]
    E, G, blocks = rp.distributed_step(pair_forces, da.Z, da.coords, rank, world, dist, costs=costs)
    out["images"] = (E.numpy(), G.numpy(), blocks)
    # more ranks than replicas: an empty block on this rank
    E, G, blocks = rp.distributed_step(pair_forces, da.Z[:1], da.coords[:1], rank, world, dist, costs=[3.0])
    out["one"] = (E.numpy(), G.numpy(), blocks)
    t = bench.max_over_ranks(1.0 + 2.0 * rank, dist, torch.device("cpu"))
    out["timing"] = (t, bench.job_throughput(4, world, 3, t))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_gather_equals_single_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    beads, da = _step_inputs()
    for key, (Z, X) in {"beads": (beads.Z, beads.coords), "images": (da.Z, da.coords),
                        "one": (da.Z[:1], da.coords[:1])}.items():
        E0, G0 = pair_forces(Z, X)
        for rank in range(world):
            E, G, blocks = res[rank][key]
            np.testing.assert_array_equal(E, E0)     # same arithmetic, gathered unchanged
            np.testing.assert_array_equal(G, G0)
            assert blocks == res[0][key][2]          # every rank derives the same split
    assert res[0]["beads"][2] == [(0, 3), (3, 5)]
    assert res[0]["one"][2] == [(0, 1), (1, 1)]
    # the image split balances the cost better than an even split of the count
    costs = [len(z) ** 4 for z in da.Z]
    bal = max(RP.block_costs(costs, res[0]["images"][2]))
    even = max(RP.block_costs(costs, RP.contiguous_blocks(len(costs), world)))
    assert bal <= even
    for rank in range(world):
        t, v = res[rank]["timing"]
        assert t == 3.0                              # max over ranks of 1.0 and 3.0
        assert v == pytest.approx(4 * 2 * 3 / 3.0)


def test_contiguous_blocks():
    assert RP.contiguous_blocks(10, 4) == [(0, 3), (3, 6), (6, 8), (8, 10)]
    assert RP.contiguous_blocks(2, 3) == [(0, 1), (1, 2), (2, 2)]
    assert RP.contiguous_blocks(0, 2) == [(0, 0), (0, 0)]


@pytest.mark.parametrize("seed", range(6))
def test_balanced_blocks_is_the_best_contiguous_split(seed):
    """Against brute force over every set of cut points (small cases)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    world = int(rng.integers(1, 5))
    costs = rng.integers(1, 50, size=n).astype(float)
    blocks = RP.balanced_blocks(costs, world)
    assert len(blocks) == world and blocks[0][0] == 0 and blocks[-1][1] == n
    assert all(blocks[i][1] == blocks[i + 1][0] for i in range(world - 1))
    best = np.inf
    for cuts in itertools.combinations_with_replacement(range(n + 1), world - 1):
        edges = (0,) + cuts + (n,)
        best = min(best, max(costs[edges[i]:edges[i + 1]].sum() for i in range(world)))
    assert max(RP.block_costs(costs, blocks)) == pytest.approx(best)


def _split_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from paper_1601_02713_gb300 import native
    from paper_1601_02713_gb300 import replicas as rp
    o = native.scf_opts(split_size=world, split_rank=rank, reduce=rp.allreduce_fn(dist, host=True))
    buf = np.arange(6, dtype=np.float64) * (rank + 1)
    # the library's call: reduce_fn(buffer address, length, user)
    rc = o.reduce_fn(buf.ctypes.data, len(buf), None)
    q.put((rank, rc, buf.tolist(), o.split_size, o.split_rank))
    dist.barrier()
    dist.destroy_process_group()


def test_force_split_reduce_callback_over_gloo():
    """The reduce function of the force-parallel split, called through the
    C function pointer the library receives: every rank's buffer becomes the
    sum over the ranks (here host buffers and gloo; NCCL and device buffers
    on GPUs)."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict((r, rest) for r, *rest in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        rc, buf, size, r = res[rank]
        assert rc == 0 and size == world and r == rank
        np.testing.assert_array_equal(buf, np.arange(6) * 3.0)


def test_reduce_callback_reports_errors():
    from paper_1601_02713_gb300 import native

    def bad(ptr, n):
        raise RuntimeError("peer lost")
    o = native.scf_opts(split_size=2, split_rank=0, reduce=bad)
    buf = np.zeros(3)
    assert o.reduce_fn(buf.ctypes.data, 3, None) == 1
