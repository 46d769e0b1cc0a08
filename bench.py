#!/usr/bin/env python
"""Benchmark of the Kryging hot path on one GB300 (or N replicas).

One step = one profile log-likelihood evaluation of the grid1024 workload plus
its kriging means: embedding eigenvalues, SLQ log-determinant (64 Rademacher
probes x 60 Lanczos steps, one batched launch sequence), CG solves of
K [y, X] (FP32 CG with FP64 residual replacement), GLS beta and loglik, and the kriging mean at
every unobserved cell.  Inputs are resident on the device before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload, scaled to the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2012_13133_gb300 import inputs as I  # noqa: E402

WORKLOAD = "grid1024"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "matvec_grid1024.md")
KERNEL_SOURCES = ["paper_2012_13133_gb300/csrc/matvec.cu", "paper_2012_13133_gb300/csrc/fft.cuh",
                  "paper_2012_13133_gb300/csrc/fft16.cuh", "paper_2012_13133_gb300/csrc/fftspec.cuh",
                  "paper_2012_13133_gb300/csrc/mvspec.cuh", "paper_2012_13133_gb300/csrc/mvspec_a.cu",
                  "paper_2012_13133_gb300/csrc/mvspec_b.cu", "paper_2012_13133_gb300/csrc/mvspec_c.cu",
                  "paper_2012_13133_gb300/csrc/kry_internal.cuh"]


def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def workload_desc(w):
    return (f"{w.name}: {w.n1}x{w.n2} grid, {int(round((1 - w.frac_missing) * 100))}% observed "
            f"({w.mask} mask), Matern nu={w.cov.nu}, range={w.cov.range}, sigma2={w.cov.sigma2}, "
            f"tau2={w.cov.tau2}; SLQ {w.nprobe} probes x {w.nsteps} Lanczos steps; CG on K[y,X] to "
            f"rel. res. {w.cg_tol:g} (FP32 CG, FP64 residual replacement); GLS beta; kriging mean at all unobserved cells")


def max_over_ranks(x, device, world):
    """Largest value of x over the ranks of the default process group (x itself when world == 1):
    every rank's timed region ends only when the slowest replica's does."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, steps, seconds):
    """Whole-job evaluations per second of world replicas that each ran steps evaluations, with
    seconds the slowest rank's time (weak scaling: the work per GPU is fixed)."""
    return world * steps / seconds


def model_bytes_per_vector(n1, n2, M1, M2, p):
    """Algorithmic bytes of the 3-pass FP32 matvec per real vector: the
    n1 x M2 complex slab written and read twice (16 n1 M2), the vector read,
    re-read for the nugget and written plus the index lists (16 p)."""
    return 16.0 * n1 * M2 + 16.0 * p


def floor_bytes_per_vector(p):
    """Compulsory bytes of one FP32 matvec per real vector if the whole 2-D
    transform stayed on chip (one pass): the vector read, the result written
    and the Krylov epilogue's two vector reads (16 p)."""
    return 16.0 * p


def read_traffic():
    """[(real vectors per launch, DRAM bytes per launch), ...] of the matvec
    from the committed ncu summary (one entry per captured batch width), if
    it was taken on the current kernel sources; None otherwise."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", txt)
    pts = [(int(a), float(b)) for a, b in re.findall(r"dram_bytes_per_launch_at_(\d+)_vectors:\s*([0-9.eE+]+)", txt)]
    if not m or not pts or m.group(1) != kernel_hash():
        return None
    return sorted(pts)


def traffic_at(points, nv):
    """DRAM bytes per launch at nv real vectors per launch: linear through the
    captured batch widths (a launch mix of two widths averages to the line at
    its mean width), proportional to nv from a single capture."""
    if len(points) == 1:
        n0, b0 = points[0]
        return b0 * nv / n0
    (n0, b0), (n1, b1) = points[0], points[-1]
    return b0 + (b1 - b0) * (nv - n0) / (n1 - n0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return self.summarise(lines)

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum SM clock and the throttle reasons seen Active in nvidia-smi CSV
        rows of FIELDS (noheader, nounits); None without a complete row."""
        rows = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# ---------------------------------------------------------------------------- GPU arm

class Problem:
    def __init__(self, ctx, w, dev):
        import torch
        from paper_2012_13133_gb300 import kry
        self.w = w
        self.mask = I.make_mask(w)
        self.mask_dev = torch.from_numpy(self.mask.astype(np.uint8)).to(dev)
        self.p = ctx.set_mask(self.mask_dev)
        S1, S2 = I.cell_centres(w.n1, w.n2)
        X = I.covariates(S1[self.mask], S2[self.mask])
        self.Xt = torch.tensor(X.T.copy(), device=dev)
        cov = w.cov
        M1, M2, _ = ctx.sample_size(cov)
        xi, eps = I.data_noise(M1, M2, self.p, w.data_seed)
        field = ctx.sample(cov, M1, M2, torch.tensor(xi, device=dev))
        beta = torch.tensor(w.beta, device=dev, dtype=torch.float64)
        self.y = (self.Xt.T @ beta + field[self.mask_dev.bool()] +
                  math.sqrt(cov.tau2) * torch.tensor(eps, device=dev)).contiguous()
        cells = np.flatnonzero(~self.mask.ravel()).astype(np.int64)
        self.cells = torch.tensor(cells, device=dev)
        self.Xc = torch.tensor(I.covariates(S1.ravel()[cells], S2.ravel()[cells]).T.copy(), device=dev)
        self.mean = torch.empty(cells.size, dtype=torch.float64, device=dev)
        self.opts = kry.Opts(prec=kry.KRY_F32, nprobe=w.nprobe, nsteps=w.nsteps, seed=w.probe_seed,
                             rtol=w.cg_tol, maxit=10000, reorth=w.reorth)
        self.M1, self.M2 = I_embed(w.n1), I_embed(w.n2)
        # host copies for the end-to-end leg (pinned)
        self.y_h = self.y.cpu().pin_memory()
        self.Xt_h = self.Xt.cpu().pin_memory()
        self.mask_h = self.mask_dev.cpu().pin_memory()
        self.cells_h = self.cells.cpu().pin_memory()
        self.Xc_h = self.Xc.cpu().pin_memory()

    def step(self, ctx):
        return ctx.loglik_krige(self.w.cov, self.opts, self.y, self.Xt, cells=self.cells, Xc=self.Xc,
                                mean_cells=self.mean)


def I_embed(n):
    M = 1
    while M < 2 * n:
        M *= 2
    return M


def flush_l2(buf):
    buf.add_(1.0)


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2012_13133_gb300 import kry

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = I.WORKLOADS[args.workload]
    ctx = kry.Context(local_rank)
    stream = torch.cuda.current_stream(local_rank)
    prob = Problem(ctx, w, dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2
    # set-up (untimed): autotune the matvec schedules for the SLQ batch and the CG batch
    emb = ctx.embed(w.cov, kry.KRY_F32)
    tuned = {str(nv): ctx.autotune(emb, nv) for nv in (w.nprobe, prob.Xt.shape[0] + 1)}
    emb.free()

    for _ in range(args.warmup):
        flush_l2(flush)
        prob.step(ctx)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = kry.launch_count()
    dev_ms = 0.0
    statuses = []
    ll_vals = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush_l2(flush)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = prob.step(ctx)
        e1.record(stream)
        e1.synchronize()
        dev_ms += e0.elapsed_time(e1)
        statuses.append(int(res["status"]))
        ll_vals.append(float(res["loglik"]))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = kry.launch_count() - launches0
    clk = clocks.stop()
    # one more step with every matvec timed by CUDA events on the context stream
    # (kry_profile_enable): the per-launch duration of the dominant kernel for
    # the roofline, kept out of the timed steps above
    flush_l2(flush)
    torch.cuda.synchronize()
    ctx.profile_enable(True)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    prob.step(ctx)
    p1.record(stream)
    p1.synchronize()
    prof_step_ms = p0.elapsed_time(p1)
    prof32 = ctx.profile_read(kry.KRY_F32)
    prof64 = ctx.profile_read(kry.KRY_F64)
    ctx.profile_enable(False)
    if world > 1:
        dist.barrier()
    dev_ms = max_over_ranks(dev_ms, dev, world)

    # ---- end to end: host buffers, H2D + D2H inside the timed region
    e2e = None
    if not args.no_e2e:
        y_d = torch.empty_like(prob.y)
        X_d = torch.empty_like(prob.Xt)
        m_d = torch.empty_like(prob.mask_dev)
        c_d = torch.empty_like(prob.cells)
        xc_d = torch.empty_like(prob.Xc)
        h2d = (prob.y_h.numel() * 8 + prob.Xt_h.numel() * 8 + prob.mask_h.numel() + prob.cells_h.numel() * 8 +
               prob.Xc_h.numel() * 8)
        d2h = 0
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            flush_l2(flush)
            y_d.copy_(prob.y_h, non_blocking=True)
            X_d.copy_(prob.Xt_h, non_blocking=True)
            m_d.copy_(prob.mask_h, non_blocking=True)
            c_d.copy_(prob.cells_h, non_blocking=True)
            xc_d.copy_(prob.Xc_h, non_blocking=True)
            ctx.set_mask(m_d)
            res = ctx.loglik_krige(w.cov, prob.opts, y_d, X_d, cells=c_d, Xc=xc_d)
            mean_h = res["mean_cells"].cpu()
            d2h = mean_h.numel() * 8 + 8 * (2 + X_d.shape[0])
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e_s = max_over_ranks(e2e_s, dev, world)
        e2e = {"value": replica_throughput(world, args.steps, e2e_s), "unit": "evals/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        return None

    value = replica_throughput(world, args.steps, dev_ms / 1000.0)
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs") if peaks else 6800.0
    peak_src = "measured" if peaks else "fallback"
    n1, n2, M1, M2, p = w.n1, w.n2, prob.M1, prob.M2, prob.p
    bytes_vec = model_bytes_per_vector(n1, n2, M1, M2, p)
    roof = None
    if prof32["calls"] > 0 and prof32["ms"] > 0:
        alg = bytes_vec * prof32["vectors"] + 4.0 * M1 * M2 * prof32["calls"]
        achieved = alg / (prof32["ms"] / 1000.0) / 1e9
        measured = read_traffic()
        per_launch_vectors = prof32["vectors"] / prof32["calls"]
        # ncu traffic per launch at this run's mean batch, from the captures at
        # the CG batch (4 vectors) and the Lanczos batch (64 vectors)
        lam_bytes = 4.0 * M1 * M2
        traffic = None
        if measured is not None:
            traffic = round(traffic_at(measured, per_launch_vectors))
        floor = floor_bytes_per_vector(p) * prof32["vectors"] + lam_bytes * prof32["calls"]
        floor_gbs = floor / (prof32["ms"] / 1000.0) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_src,
                "floor_achieved": round(floor_gbs, 1), "frac_floor": round(floor_gbs / peak, 4),
                "floor_model": "16 p bytes per real vector + 4 M1 M2 eigenvalue bytes per launch (single pass)",
                "timing": "every FP32 matvec of one extra instrumented step (CUDA events on the context stream); "
                          "the timed steps run uninstrumented",
                "traffic": traffic,
                "kernel": "FP32 3-pass FFT matvec (passes A+B+C of one call)",
                "launches": prof32["calls"], "mean_vectors_per_launch": round(per_launch_vectors, 2),
                "mean_launch_ms": round(prof32["ms"] / prof32["calls"], 4),
                "algorithmic_bytes_per_launch": round(alg / prof32["calls"]),
                "share_of_step": round(prof32["ms"] / prof_step_ms, 3),
                "fp64_matvec_share_of_step": round(prof64["ms"] / prof_step_ms, 3),
                "instrumented_step_ms": round(prof_step_ms, 3)}

    out = {
        "metric": "profile-loglik evals/s",
        "value": round(value, 4),
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dev_ms / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_desc(w), "grid": [n1, n2], "embedding": [M1, M2], "p": p,
                   "probes": w.nprobe, "lanczos_steps": w.nsteps,
                   "lanczos_basis": "partial reorthogonalisation" if w.reorth else "plain recurrence",
                   "kriging_cells": int(prob.cells.numel()),
                   "l2": "flushed between steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "gpu_launches": int(launches),
        "library_launches_before_timed": int(launches0),
        "clocks": clk,
        "e2e": e2e,
        "wall_s": round(wall, 3),
        "loglik": ll_vals[-1],
        "status": statuses[-1],
        "tuned_schedules": tuned,
    }
    if world == 1 and not args.no_cpu_baseline:
        mv_step = prof32["vectors"] + prof64["vectors"]
        out["real_vector_matvecs_per_step"] = round(mv_step)
        out["cpu_baseline"] = cpu_baseline(w, mask=prob.mask, mv_per_eval=mv_step, budget_s=args.cpu_budget)
    return out


# ---------------------------------------------------------------------------- CPU oracle arm

def matvecs_per_eval(w, measured=None):
    """Real-vector matvecs of one evaluation.  `measured` is the count the GPU
    run made per step (SLQ probes x steps, every CG iteration on each
    right-hand side, true-residual and kriging matvecs); without it, the SLQ
    part plus 2500 CG iterations on each of the 4 right-hand sides (the count
    measured for this workload on GB300) and one kriging matvec."""
    if measured:
        return int(round(measured))
    return w.nprobe * w.nsteps + 4 * 2500 + 1


def cpu_baseline(w, mask=None, mv_per_eval=None, budget_s=20.0):
    """Time the oracle's FP64 FFT matvec inside its Lanczos loop on the full
    workload (one probe, up to nsteps steps or ~budget_s seconds), and scale
    to evaluations/s by the real-vector matvecs of one evaluation."""
    from oracle import kryoracle as O
    if mask is None:
        mask = I.make_mask(w)
    P = O.FFTProblem(w.n1, w.n2, mask, w.cov)
    z = O.rademacher_probe(w.probe_seed, 0, P.p)
    n = 0
    t0 = time.perf_counter()
    q = z / np.linalg.norm(z)
    while n < w.nsteps and (time.perf_counter() - t0) < budget_s:
        q = P.matvec(q)
        q /= np.linalg.norm(q)
        n += 1
    t = time.perf_counter() - t0
    per_mv = t / n
    mpe = matvecs_per_eval(w, mv_per_eval)
    evals = 1.0 / (per_mv * mpe)
    # the same loop on one core (the oracle's FFTs with one worker), a shorter sample
    workers = O._WORKERS
    O._WORKERS = 1
    n1c = 0
    t0 = time.perf_counter()
    q = z / np.linalg.norm(z)
    while n1c < w.nsteps and (time.perf_counter() - t0) < max(1.0, budget_s / 4):
        q = P.matvec(q)
        q /= np.linalg.norm(q)
        n1c += 1
    per_mv1 = (time.perf_counter() - t0) / n1c
    O._WORKERS = workers
    return {"value": evals, "unit": "evals/s", "cores": workers, "kind": "oracle",
            "one_core": {"value": 1.0 / (per_mv1 * mpe), "ms_per_matvec": round(per_mv1 * 1e3, 1),
                         "matvecs_timed": n1c},
            "sample": f"{n} FP64 FFT matvecs of the oracle at full size ({per_mv * 1e3:.1f} ms each, one real "
                      f"vector each, inside its Lanczos loop; the vector updates and reorthogonalisation of the "
                      f"full method are not counted), scaled by {mpe} real-vector matvecs per evaluation "
                      f"({'as counted in the GPU step' if mv_per_eval else 'SLQ + 4 x 2500 CG iterations + 1'})"}


def run_reference(args, rank):
    if rank != 0:
        return None
    w = I.WORKLOADS[args.workload]
    mask = I.make_mask(w)
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    vals = []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(w, mask=mask, budget_s=budget)
        if k >= args.warmup:
            vals.append(cb["value"])
    value = statistics.mean(vals)
    return {"metric": "profile-loglik evals/s", "value": value, "unit": "evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_desc(w)},
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(I.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
