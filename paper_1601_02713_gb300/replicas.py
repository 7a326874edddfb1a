"""Replica parallelism over several GPUs (one process per GPU).

The paper (Sec. 2, Fig. 1) splits the replicas of a step (PIMD beads or
string images) over groups of processes; every group computes the
Born-Oppenheimer energies and forces of its replicas and the results of all
groups are combined with one collective at the end of the step (an
all-reduce of zero-padded arrays), after which every process holds every
replica's energy and forces for the step of the replica dynamics.

Here each rank owns one GPU and one contiguous block of the step's replicas:
* beads of one molecule: blocks of equal size (sizes differ by at most one);
* string images of different sizes: blocks balanced by the estimated cost of
  each image, its screened shell-quartet count (pimd_screened_quartets), so
  that the slowest rank finishes as early as a contiguous split allows
  (the paper's load imbalance across images, Sec. 3.2);
then one all-gather of the energies and gradients (zero-padded to the largest
block, the paper's padded all-reduce written as an all-gather). Nothing is
exchanged during the SCF. The collective goes through torch.distributed
(NCCL between GPUs, gloo on CPU ranks in the tests).
"""
from __future__ import annotations

import numpy as np


def contiguous_blocks(n: int, world: int) -> list[tuple[int, int]]:
    """[start, end) of each rank's block of n replicas: contiguous, sizes
    differing by at most one, the larger blocks first."""
    if n < 0 or world < 1:
        raise ValueError("bad sizes")
    base, extra = divmod(n, world)
    out, s = [], 0
    for r in range(world):
        e = s + base + (1 if r < extra else 0)
        out.append((s, e))
        s = e
    return out


def balanced_blocks(costs, world: int) -> list[tuple[int, int]]:
    """Contiguous split of replicas with the given costs over `world` ranks
    that minimises the largest block cost (binary search over the bound, a
    greedy left-to-right fill decides each bound; exact for positive costs).
    Empty blocks are allowed when there are fewer replicas than ranks."""
    c = np.asarray(costs, dtype=np.float64)
    n = len(c)
    if world < 1 or np.any(c < 0):
        raise ValueError("bad costs or world size")
    if n == 0:
        return [(0, 0)] * world

    def fill(bound):
        blocks, s, acc = [], 0, 0.0
        for i in range(n):
            if acc > 0 and acc + c[i] > bound:
                blocks.append((s, i))
                s, acc = i, 0.0
            acc += c[i]
        blocks.append((s, n))
        return blocks

    lo, hi = float(c.max()), float(c.sum())
    for _ in range(100):
        if hi - lo <= 1e-9 * max(hi, 1.0):
            break
        mid = 0.5 * (lo + hi)
        if len(fill(mid)) <= world:
            hi = mid
        else:
            lo = mid
    blocks = fill(hi)
    while len(blocks) < world:
        blocks.append((n, n))
    return blocks


def block_costs(costs, blocks) -> list[float]:
    c = np.asarray(costs, dtype=np.float64)
    return [float(c[s:e].sum()) for s, e in blocks]


def gather_results(E_local, G_local, blocks, atom_counts, dist, device=None):
    """All-gather of one step's results: every rank passes its block's
    energies [n_r] and gradients [sum of its replicas' atoms, 3] (beads: any
    shape whose leading entries are per replica); returns (E [n], G [sum of
    all atoms, 3]) in replica order on every rank. blocks: each rank's
    [start, end); atom_counts: atoms of every replica of the step. The blocks
    are zero-padded to the largest one, so one collective of one size moves
    them (the paper's padded reduction)."""
    import torch
    world = len(blocks)
    atoms = np.asarray(atom_counts, dtype=np.int64)
    nmax = max(e - s for s, e in blocks)
    amax = max(int(atoms[s:e].sum()) for s, e in blocks)
    dev = device if device is not None else torch.device("cpu")
    E_local = torch.as_tensor(np.asarray(E_local, dtype=np.float64) if not torch.is_tensor(E_local) else E_local,
                              dtype=torch.float64, device=dev).reshape(-1)
    G_local = torch.as_tensor(np.asarray(G_local, dtype=np.float64) if not torch.is_tensor(G_local) else G_local,
                              dtype=torch.float64, device=dev).reshape(-1, 3)
    buf = torch.zeros(nmax + 3 * amax, dtype=torch.float64, device=dev)
    buf[:E_local.numel()] = E_local
    buf[nmax:nmax + G_local.numel()] = G_local.reshape(-1)
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    Es, Gs = [], []
    for (s, e), p in zip(blocks, parts):
        na = int(atoms[s:e].sum())
        Es.append(p[:e - s])
        Gs.append(p[nmax:nmax + 3 * na].reshape(na, 3))
    return torch.cat(Es), torch.cat(Gs)


def distributed_step(forces_fn, Z_list, coords_list, rank: int, world: int, dist, costs=None, device=None):
    """One force step of all replicas split over the ranks: rank `rank`
    evaluates its block with forces_fn(Z_block, coords_block) -> (E [n_r],
    G [sum atoms, 3]) and the results of all ranks are gathered. costs: per
    replica (string images: screened-quartet counts); None splits evenly.
    Returns (E [n], G [sum atoms, 3], blocks) on every rank."""
    n = len(Z_list)
    blocks = contiguous_blocks(n, world) if costs is None else balanced_blocks(costs, world)
    s, e = blocks[rank]
    atoms = [len(z) for z in Z_list]
    if e > s:
        E_loc, G_loc = forces_fn(Z_list[s:e], coords_list[s:e])
    else:
        E_loc, G_loc = np.zeros(0), np.zeros((0, 3))
    E, G = gather_results(E_loc, G_loc, blocks, atoms, dist, device)
    return E, G, blocks


# ---------------------------------------------------------------------------
# Force-parallel split of each replica (the paper's force groups, Sec. 2):
# m processes share every replica's quartet tiles and sum their partial Fock
# matrices (and two-electron gradients) after every build. The library calls
# a reduce function with a device buffer; these build one.
# ---------------------------------------------------------------------------
class _DeviceView:
    """A float64 device buffer (address, length) as a CUDA array interface,
    so that torch can view it without a copy."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_view(ptr: int, n: int):
    import torch
    return torch.as_tensor(_DeviceView(ptr, n), device="cuda")


def host_view(ptr: int, n: int):
    """A float64 host buffer (address, length) as a torch tensor (no copy)."""
    import ctypes
    import torch
    a = np.ctypeslib.as_array(ctypes.cast(int(ptr), ctypes.POINTER(ctypes.c_double)), shape=(int(n),))
    return torch.from_numpy(a)


def allreduce_fn(dist, group=None, host=False):
    """reduce function for native.scf_opts(split_size=m, split_rank=r,
    reduce=...): an in-place all-reduce (sum) of the library's device buffer
    over the process group (NCCL), finished before it returns. host=True
    treats the address as host memory (gloo process groups)."""
    import torch

    def fn(ptr, n):
        t = host_view(ptr, n) if host else device_view(ptr, n)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        if not host:
            torch.cuda.synchronize()
    return fn


class ThreadSum:
    """reduce functions for m host threads that share one GPU (one context
    each): every call deposits a host copy of its buffer, waits for the
    others (a host barrier; no kernel waits on another) and writes the sum
    back. The threads must make their calls in the same order."""

    def __init__(self, m: int, timeout: float = 300.0):
        import threading
        self.m = m
        # a thread that left its forces call (an error) breaks the barrier
        # after the timeout instead of leaving the others waiting
        self.bar = threading.Barrier(m, timeout=timeout)
        self.parts = [None] * m

    def fn(self, rank: int):
        import torch

        def f(ptr, n):
            t = device_view(ptr, n)
            self.parts[rank] = t.cpu()
            self.bar.wait()
            total = sum(self.parts[1:], self.parts[0].clone())
            self.bar.wait()
            t.copy_(total.to(t.device))
            torch.cuda.synchronize()
        return f
