#!/usr/bin/env python
"""Benchmark: RHF bead energy+gradient evaluations per second on GB300.

One step = one `pimd_bo_forces_dev` call over every bead of one PIMD step
(the paper's force step, Sec. 2): the whole hot path (integrals, SCF to
|dE| < 1e-10 Eh and max|e| < 1e-8, analytic gradient) for all beads in the
same launches. Consecutive steps move every atom by a Gaussian displacement
(sigma/sqrt(10) of the bead jitter), like consecutive MD steps, and each step
starts from the previous step's MOs of the same bead (Sec. 2: MOs kept in
memory and reused as the next step's guess).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun the step's replicas are split over the ranks, one GPU each
(Sec. 2: replica parallelism): beads in equal contiguous blocks, the step
holding world x (beads per rank) beads (weak scaling); string images, whose
number is fixed by the workload, in contiguous blocks balanced by their
screened-quartet counts (strong scaling). After its forces call every rank
takes part in one all-gather of all replicas' energies and gradients (the
paper's gather of forces before the replicas move), inside the timed step.
The step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1601_02713_gb300 import inputs  # noqa: E402

METRIC = "RHF bead energy+gradient evals/sec at stated accuracy; Fock-build GERI/s"
UNIT = "bead evals/s"
# FP64 pipe of GB300: 4 FP64 flops per clock per SM (2 FMA; the FMA-chain
# microbenchmark measured 1.255 TFLOP/s), 152 SMs, 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
# FP32 pipe: 128 FP32 lanes x 2 flops (FMA) per clock per SM (the FMA-chain
# microbenchmark measured 76.7 TFLOP/s)
FP32_PEAK_TFLOPS = 152 * 256 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="water8_spd_32beads")
    ap.add_argument("--nrep", type=int, default=None, help="beads per rank (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-quartets", type=int, default=100000)
    ap.add_argument("--cpu-sample-deriv", type=int, default=8000)
    ap.add_argument("--fp32-tau", type=float, default=0.0,
                    help="mixed precision: quartets with Q_ab Q_cd max|dD| below this run in FP32 (0: all FP64)")
    ap.add_argument("--prim-screen", type=float, default=None,
                    help="primitive-quartet cutoff as a fraction of the quartet cutoff (default: the library's 1/81)")
    ap.add_argument("--ref-iterations", type=float, default=15.3,
                    help="reference arm: SCF iterations per bead evaluation used to scale the oracle sample")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default kernels (straight-line, 128-quartet tiles) instead of tuning them")
    ap.add_argument("--guess-study", action="store_true",
                    help="instead of the benchmark line: train the learned density guess on the GPU and compare "
                         "SCF iterations and evals/s of the guesses (one JSON line)")
    ap.add_argument("--train-clusters", type=int, default=8)
    ap.add_argument("--train-beads", type=int, default=16)
    ap.add_argument("--train-epochs", type=int, default=400)
    ap.add_argument("--eval-water32", type=int, default=0,
                    help="guess study: also start this many (H2O)32 beads (mixed precision) from SAD and from the "
                         "learned density")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------- inputs
def make_steps(name, nrep, nsteps, world=1):
    """The job's steps (every rank builds the same sequence): for beads of
    one molecule, world x nrep beads per step (nrep: beads per rank, default
    the workload's); string images as the workload defines them."""
    reps, kind = inputs.workload(name, nrep=nrep)
    if reps.uniform() and world > 1:
        reps, kind = inputs.workload(name, nrep=len(reps.Z) * world)
    seq = inputs.markov_steps(reps, nsteps, seed=97)
    return seq, kind


def rank_block(seq, blocks, rank):
    """This rank's contiguous block of replicas of every step."""
    s, e = blocks[rank]
    return [inputs.Replicas(st.Z[s:e], st.coords[s:e], st.name) for st in seq]


def max_over_ranks(t_local, dist, device):
    """Step time of the whole job: the maximum over ranks (every rank waits
    for the slowest before the next step)."""
    if dist is None:
        return t_local
    import torch
    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(beads_per_rank, world, steps, t_max):
    """Whole-job bead evaluations per second: all ranks' beads over the
    slowest rank's time (beads: each rank evaluates its own block of the step)."""
    return beads_per_rank * world * steps / t_max


# ---------------------------------------------------------------- CPU baseline (oracle)
def oracle_whole(step_reps, kind):
    """The oracle on every replica of the step, whole: one-electron integrals,
    SCF to the same bars, gradient (small systems). Returns (replica evals/s,
    threads, sample text, s)."""
    import oracle as O
    bas = inputs.basis_set(kind)
    t0 = time.time()
    for Z, X in zip(step_reps.Z, step_reps.coords):
        O.rhf_energy_gradient(bas, Z, X)
    dt = time.time() - t0
    n = len(step_reps.Z)
    return n / dt, O.num_threads(), f"every replica of the step ({n}), whole: integrals, SCF and gradient", dt


def oracle_sample(step_reps, kind, iterations, n_eri, n_der, seed=11):
    """Time the oracle on a bounded sample of one bead of the workload:
    random screened shell quartets of bead 0 for the Fock build (n_eri) and for
    the derivative integrals (n_der); per-bead time = iterations x quartets x
    t_eri + quartets x t_der. Systems of at most 64 basis functions are timed
    whole instead (oracle_whole). Returns (bead evals/s, threads, sample
    text, s)."""
    import oracle as O
    bas = inputs.basis_set(kind)
    Z, X = step_reps.Z[0], step_reps.coords[0]
    ob = O.OracleBasis.build(bas, Z, X)
    if ob.nbf <= 64:
        return oracle_whole(step_reps, kind)
    t0 = time.time()
    q = O.canonical_quartets(ob, 1e-12)
    rng = np.random.default_rng(seed)
    se = q[rng.choice(len(q), min(n_eri, len(q)), replace=False)]
    sd = q[rng.choice(len(q), min(n_der, len(q)), replace=False)]
    t = time.time()
    O.eri_list(ob, se)
    te = (time.time() - t) / len(se)
    t = time.time()
    O.deriv_list(ob, sd)
    td = (time.time() - t) / len(sd)
    per_bead = len(q) * (iterations * te + td)
    sample = (f"bead 0 of the first timed step: {len(se)} of its {len(q)} screened shell quartets timed for the "
              f"Fock build and {len(sd)} for the derivative integrals; per-bead time = {iterations:.1f} Fock builds "
              f"(the GPU's mean per bead) x {len(q)} x {te * 1e6:.1f} us + {len(q)} x {td * 1e6:.1f} us = "
              f"{per_bead:.0f} s")
    return 1.0 / per_bead, O.num_threads(), sample, time.time() - t0


def run_reference(args):
    """The oracle as the reference arm: each step is the bounded oracle sample
    of the same workload, reported in the same unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    seq, kind = make_steps(args.workload, args.nrep, 1)
    # SCF iterations per bead evaluation: the mean the GPU path measures on
    # this workload (15.3 for (H2O)8 with MO reuse between steps)
    iters = args.ref_iterations
    vals = []
    n_eri = max(1000, args.cpu_sample_quartets // 4)
    n_der = max(200, args.cpu_sample_deriv // 4)
    for s in range(args.warmup + args.steps):
        v, thr, sample, secs = oracle_sample(seq[0], kind, iters, n_eri, n_der, seed=100 + s)
        if s >= args.warmup:
            vals.append(v)
    value = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(seq[0].Z) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "beads_per_rank": len(seq[0].Z), "basis": kind,
                       "iterations_assumed": iters},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- learned-guess study
def run_guess_study(args):
    """Train the learned density guess on converged (H2O)8 bead densities
    (seeded clusters other than the benchmark's, mixed-precision SCF), then run
    the benchmark's beads (energy + gradient) from each starting guess and in
    each form: plain per-bead FP64 calls (SAD guess), batched FP64 (core,
    SAD, learned, previous-step MOs) and batched mixed precision (learned,
    previous-step MOs). Reports SCF iterations, bead evals/s and the largest
    energy and gradient deviation from the batched FP64 SAD run."""
    import torch
    from paper_1601_02713_gb300 import build as B
    B.build()
    from paper_1601_02713_gb300 import native
    torch.cuda.set_device(0)
    seq, kind = make_steps(args.workload, args.nrep, 2)
    Z, X0 = seq[0].stacked()
    _, X1 = seq[1].stacked()
    nrep = len(X0)
    basis = native.Basis(inputs.basis_set(kind))
    ctx = native.Context(0)
    model = native.GuessModel(basis, seed=5)
    t0 = time.perf_counter()
    ntrain = 0
    for reps in inputs.water_cluster_set(len(Z) // 3, args.train_clusters, args.train_beads, 500):
        Zt, Xt = reps.stacked()
        model.add_data(ctx, basis, Zt, Xt, native.scf_opts(guess=4, fp32_tau=1e-6, want_gradient=0))
        ntrain += len(Xt)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = model.train(args.train_epochs, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    model.attach(ctx)

    def run(X, guess, fp32_tau, per_bead=False):
        torch.cuda.synchronize()
        t = time.perf_counter()
        if per_bead:
            out = [native.pimd_bo_forces(ctx, basis, Z, X[i:i + 1], native.scf_opts(guess=guess, fp32_tau=fp32_tau))
                   for i in range(len(X))]
            E = np.concatenate([o[0] for o in out])
            G = np.concatenate([o[1] for o in out])
            info = [o[2][0] for o in out]
        else:
            E, G, info, _ = native.pimd_bo_forces(ctx, basis, Z, X, native.scf_opts(guess=guess, fp32_tau=fp32_tau))
        dt = time.perf_counter() - t
        assert all(i["converged"] for i in info)
        return E, G, float(np.mean([i["iterations"] for i in info])), len(X) / dt

    rows = []
    ctx.clear_guess()
    Eref, Gref, it, v = run(X0, 4, 0.0)
    rows.append(("batched", "fp64", "SAD", it, v, Eref, Gref))
    for form, prec, guess, tau, per in [("per-bead", "fp64", "SAD", 0.0, True), ("batched", "fp64", "core", 0.0, False),
                                        ("batched", "fp64", "learned", 0.0, False),
                                        ("batched", "mixed", "learned", 1e-6, False)]:
        ctx.clear_guess()
        g = {"SAD": 4, "core": 0, "learned": 2}[guess]
        E, G, it, v = run(X0, g, tau, per)
        rows.append((form, prec, guess, it, v, E, G))
    # previous-step MOs: converge the step before, then time the step
    for prec, tau in [("fp64", 0.0), ("mixed", 1e-6)]:
        ctx.clear_guess()
        run(X0, 4, tau)
        E1, G1, it, v = run(X1, 1, tau)
        rows.append(("batched", prec, "previous-step MOs (next MD step)", it, v, None, None))
    if args.eval_water32 > 0:
        reps32, _ = inputs.workload("water32_spd_16beads", nrep=args.eval_water32)
        Z32, X32 = reps32.stacked()
        for guess, gname in ((4, "SAD"), (2, "learned")):
            ctx.clear_guess()
            torch.cuda.synchronize()
            t = time.perf_counter()
            E, G, info, _ = native.pimd_bo_forces(ctx, basis, Z32, X32, native.scf_opts(guess=guess, fp32_tau=1e-6))
            dt = time.perf_counter() - t
            assert all(i["converged"] for i in info)
            it = float(np.mean([i["iterations"] for i in info]))
            rows.append(("batched (H2O)32", "mixed", gname, it, len(X32) / dt, None, None))
    out = {"study": "learned SCF guess", "workload": args.workload, "beads": nrep, "basis": kind,
           "training": {"geometries": ntrain, "system": f"(H2O){len(Z) // 3} seeded clusters 500..",
                        "data_s": t_data, "epochs": args.train_epochs, "train_s": t_train,
                        "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
           "rows": []}
    for form, prec, guess, it, v, E, G in rows:
        r = {"form": form, "precision": prec, "guess": guess, "scf_iterations_mean": it, "bead_evals_per_s": v}
        if E is not None:
            r["max_abs_dE_vs_fp64_sad"] = float(np.abs(E - Eref).max())
            r["max_abs_dG_vs_fp64_sad"] = float(np.abs(G - Gref).max())
        out["rows"].append(r)
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


# ---------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.guess_study:
        return run_guess_study(args)
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1601_02713_gb300 import build as B
    B.build()
    from paper_1601_02713_gb300 import native

    K, W, E2E = args.steps, args.warmup, args.e2e_steps
    from paper_1601_02713_gb300 import replicas as RP
    seq_all, kind = make_steps(args.workload, args.nrep, W + K + E2E, world)
    ragged = not seq_all[0].uniform()
    ctx = native.Context(local)
    basis = native.Basis(inputs.basis_set(kind))
    n_all = len(seq_all[0].Z)
    atoms_all = [len(z) for z in seq_all[0].Z]
    if ragged and world > 1:
        # string images: contiguous blocks balanced by screened-quartet counts
        nat0, Z0, X0 = seq_all[0].concat()
        costs = native.pimd_screened_quartets(ctx, basis, nat0, Z0, X0)
        blocks = RP.balanced_blocks(costs, world)
    else:
        blocks = RP.contiguous_blocks(n_all, world)
    seq = rank_block(seq_all, blocks, rank)
    nrep = len(seq[0].Z)
    # beads of one molecule (pimd_bo_forces) or string images of different
    # sizes (string_images_forces, one ragged batch)
    if ragged:
        nat, Z, _ = seq[0].concat()
        natom = int(nat.sum())
    else:
        Z, _ = seq[0].stacked()
        natom = len(Z)
    opts = native.scf_opts(guess=1, fp32_tau=args.fp32_tau)
    if args.prim_screen is not None:
        opts.prim_screen = args.prim_screen
    dev = torch.device("cuda", local)
    X = [torch.tensor(s.concat()[2] if ragged else s.stacked()[1], dtype=torch.float64, device=dev) for s in seq]
    E = torch.empty(nrep, dtype=torch.float64, device=dev)
    G = torch.empty((natom, 3) if ragged else (nrep, natom, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (126 MB)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def step(i):
        if nrep == 0:
            infos = []
        elif ragged:
            infos, rc = native.string_images_forces_dev(ctx, basis, nat, Z, X[i], E, G, opts,
                                                        stream=stream.cuda_stream)
        else:
            infos, rc = native.pimd_bo_forces_dev(ctx, basis, Z, X[i], E, G, opts, stream=stream.cuda_stream)
        if nrep and rc != 0:
            raise RuntimeError(f"forces call returned {rc}")
        if dist is not None:
            # every rank gets every replica's energy and gradient (one all-gather)
            RP.gather_results(E, G, blocks, atoms_all, dist, dev)
        return infos

    # autotuner (not timed): kernel variants for this workload (replicas of
    # one molecule; a ragged batch keeps the defaults)
    t_tune = time.perf_counter()
    widths, grad_var, tune_ms = (None, None, None) if (args.no_autotune or ragged) else \
        native.pimd_autotune(ctx, basis, Z, seq[0].stacked()[1], opts)
    t_tune = time.perf_counter() - t_tune
    ctx.clear_guess()
    for i in range(W):
        step(i)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, stats, iters = [], [], []
    for i in range(W, W + K):
        flush.zero_()
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = step(i)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms.append(e0.elapsed_time(e1))
        if nrep:
            stats.append(native.pimd_last_stats(ctx))
            iters.append(float(np.mean([x["iterations"] for x in infos])))
        assert all(x["converged"] for x in infos)
    clk = clocks.stop()
    t_local = sum(ms) / 1000.0
    t_max = max_over_ranks(t_local, dist, dev)
    # whole job: every replica of the step (all ranks' blocks) per step
    value = n_all * K / t_max

    # end to end through the host-buffer entry point (H2D coords, D2H E and G)
    # the step inputs in pinned host memory (the H2D copy is part of the call)
    Xh = []
    for i in range(W + K, W + K + E2E):
        x = seq[i].concat()[2] if ragged else seq[i].stacked()[1]
        xp = torch.empty(x.shape, dtype=torch.float64, pin_memory=torch.cuda.is_available()).numpy()
        xp[...] = x
        Xh.append(xp)
    barrier()
    t0 = time.perf_counter()
    for x in Xh:
        if nrep == 0:
            Eh, Gh = np.zeros(0), np.zeros((0, 3))
        elif ragged:
            Eh, Gh, info_h, rc = native.string_images_forces(ctx, basis, nat, Z, x, opts)
            assert rc == 0
        else:
            Eh, Gh, info_h, rc = native.pimd_bo_forces(ctx, basis, Z, x, opts)
            assert rc == 0
        if dist is not None:
            RP.gather_results(Eh, Gh, blocks, atoms_all, dist, dev)
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = n_all * E2E / t_e2e

    # roofline of the dominant kernel (the Fock build: all quartet classes)
    fock_ms = max(sum(s["ms_fock"] for s in stats), 1e-9)
    builds = sum(s["fock_builds"] for s in stats)
    flops = sum(s["eri_flops_per_build"] * s["fock_builds"] for s in stats)
    flops32 = sum(s["eri_flops32_per_build"] * s["fock_builds"] for s in stats)
    eris = sum(s["eris_per_build"] * s["fock_builds"] for s in stats)
    achieved = flops / (fock_ms * 1e-3) / 1e12
    geri = eris / (fock_ms * 1e-3) / 1e9
    eris32 = sum(s.get("eris32_per_build", 0.0) * s["fock_builds"] for s in stats)
    launches = int(sum(s["kernel_launches"] for s in stats))
    grad_ms = max(sum(s["ms_grad2e"] for s in stats), 1e-9)
    gflops = sum(s.get("grad_flops", 0.0) for s in stats)
    gflops32 = sum(s.get("grad_flops32", 0.0) for s in stats)

    Bq = native.Basis(inputs.basis_set(kind))
    if ragged:
        nbfs = [Bq.nbf(z) for z in seq[0].Z]
        basis_txt = f"{kind} (even-tempered, {min(nbfs)}-{max(nbfs)} functions per image)"
        coord_bytes = natom * 3 * 8
    else:
        basis_txt = f"{kind} (even-tempered, {Bq.nbf(Z)} functions)"
        coord_bytes = nrep * natom * 3 * 8
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_max * 1000.0 / K, "higher_is_better": True,
            "scaling": "strong" if ragged else "weak", "vs_baseline": None,
            "dtype": "f64" if args.fp32_tau == 0 else "f64+f32", "data": "synthetic",
            "config": {"workload": args.workload, "beads_per_rank": nrep, "replicas_per_step": n_all,
                       "rank_blocks": blocks,
                       "atoms": natom if not ragged else f"{min(len(z) for z in seq[0].Z)}-"
                                                         f"{max(len(z) for z in seq[0].Z)} per image",
                       "basis": basis_txt,
                       "scf": "|dE|<1e-10, max|FDS-SDF|<1e-8, DIIS(8), MO reuse between steps",
                       "schwarz_tau": 1e-12, "fp32_tau": args.fp32_tau, "prim_screen": opts.prim_screen,
                       "l2": "flushed before every timed step (512 MB write)",
                       "parallelism": f"replicas{world}"},
            "geri_per_s": geri,
            "geri_per_s_split": {"fp64": (eris - eris32) / (fock_ms * 1e-3) / 1e9,
                                 "fp32": eris32 / (fock_ms * 1e-3) / 1e9,
                                 "note": "unique contracted ERIs of each path over the whole Fock-build time"},
            "fp32_quartet_fraction": (sum(s["quartets_fp32"] for s in stats)
                                      / max(1, sum(s["quartets_fp32"] + s["quartets_fp64"] for s in stats))),
            "fock_builds_per_step": builds / K,
            "ms_split_per_step": {"fock": fock_ms / K, "grad2e": sum(s["ms_grad2e"] for s in stats) / K,
                                  "other": (t_local * 1000.0 - fock_ms - sum(s["ms_grad2e"] for s in stats)) / K},
            "eri_flops32_per_step": sum(s["eri_flops32_per_build"] * s["fock_builds"] for s in stats) / K,
            "scf_iterations_mean": statistics.mean(iters) if iters else None,
            "roofline": {"kernel": "jk_kernel (one Fock build = all quartet classes)", "bound": "alu",
                         "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "fp32_achieved": flops32 / (fock_ms * 1e-3) / 1e12,
                         "fp32_frac": flops32 / (fock_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                         "note": ("achieved/frac: FP64 operations of the Fock build over its time against the FP64 "
                                  "pipe; fp32_*: the FP32 quartets' operations over the same time against the FP32 "
                                  "pipe (mixed mode); their sum is the share of the two pipes' peak the build uses"),
                         "flops_per_launch": flops / max(builds, 1), "ms_per_launch": fock_ms / max(builds, 1),
                         "peak_source": "FP64 pipe: 152 SMs x 4 flop/clk x 2.07 GHz (FMA chain measured 1.255)"},
            "grad_roofline": {"kernel": "grad2e_kernel / grad2e_coop_kernel (all quartet classes, one per "
                                        "forces call)", "bound": "alu",
                              "achieved": gflops / (grad_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": gflops / (grad_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                              "fp32_achieved": gflops32 / (grad_ms * 1e-3) / 1e12,
                              "fp32_frac": gflops32 / (grad_ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                              "flops_per_step": gflops / K, "ms_per_step": grad_ms / K,
                              "note": ("per executed primitive quartet: the generated recursion to order L + 1 with "
                                       "its four accumulated sets, set-up and Boys; the HRRs, the density "
                                       "contraction and the Cartesian/spherical transforms are not counted")},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(coord_bytes),
                    "d2h_bytes_per_step": int(nrep * 8 + coord_bytes)},
            "gpu_launches": launches,
            "autotune": {"fock_kernel": widths, "grad_kernel": grad_var, "fock_build_ms": tune_ms,
                         "seconds": t_tune,
                         "note": ("per class pair, picked before the warm-up (not timed): Fock ket-tile width "
                                  "32/64/128 or 0 = cooperative kernel; gradient 0 = cooperative, "
                                  "1 = straight-line")},
            "clocks": clk}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, thr, sample, secs = oracle_sample(seq[W], kind, statistics.mean(iters), args.cpu_sample_quartets,
                                             args.cpu_sample_deriv)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
