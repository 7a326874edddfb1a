"""The multi-rank benchmark path on CPU ranks (gloo, world size 2): each
rank owns its own beads (no data-path collective), the step time is the
maximum over ranks, and the throughput counts every rank's beads."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench
    seq, kind = bench.make_steps("water2_min_4beads", 4, 2, rank)
    x = torch.tensor(seq[0].stacked()[1])
    xs = [torch.zeros_like(x) for _ in range(world)]
    dist.all_gather(xs, x)
    t = bench.max_over_ranks(1.0 + 2.0 * rank, dist, torch.device("cpu"))
    v = bench.job_throughput(4, world, 3, t)
    q.put((rank, float((xs[0] - xs[1]).abs().max()), t, v, kind))
    dist.barrier()
    dist.destroy_process_group()


def test_two_cpu_ranks_shard_beads_and_take_the_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dx, t, v, kind in out:
        assert dx > 1e-3          # the ranks' beads differ
        assert t == 3.0           # max over ranks of 1.0 and 3.0
        assert v == pytest.approx(4 * 2 * 3 / 3.0)
        assert kind == "min_sp"
