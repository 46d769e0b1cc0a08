"""Profiling driver for the covariance matvec kernels and the CG loop.

Sets up one workload (mask, FP32 embedding), then issues `--reps` calls of
kry_matvec on `--nvec` vectors and prints the mean CUDA-event time per call and
the model bytes per call.  With `--cg-iters N` it instead runs `--reps` CG
solves of `--nvec` right-hand sides stopped after N iterations (a tolerance no
solve reaches) and prints the time per iteration.  Small and self-contained so
that an ncu capture of its kernels ends quickly, e.g.

  ncu --set full --clock-control none -k regex:ks_pass -c 3 \
      python -m paper_2012_13133_gb300.profile_matvec --workload grid1024 --nvec 8 --reps 2
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    from paper_2012_13133_gb300 import inputs as I
    from paper_2012_13133_gb300 import kry

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="grid1024", choices=sorted(I.WORKLOADS))
    ap.add_argument("--nvec", type=int, default=8)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--autotune", action="store_true", help="autotune the schedule for this batch first")
    ap.add_argument("--sched", default="", help="fixed schedule 'rows,cols,pairs' per block/batch (no autotune)")
    ap.add_argument("--cg-iters", type=int, default=0, help="time CG iterations instead of matvec calls")
    args = ap.parse_args()

    w = I.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    ctx = kry.Context(0)
    mask = I.make_mask(w)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(dev))
    prec = kry.KRY_F32 if args.prec == "f32" else kry.KRY_F64
    dt = torch.float32 if args.prec == "f32" else torch.float64
    emb = ctx.embed(w.cov, prec)
    tuned = ctx.autotune(emb, args.nvec) if args.autotune else None
    if args.sched:
        g, c, ppb = (int(x) for x in args.sched.split(","))
        ctx.set_schedule(emb, args.nvec, g, c, ppb)
        tuned = {"rows_per_block": g, "cols_per_block": c, "pairs_per_batch": ppb}
    if args.cg_iters:
        B = torch.tensor(I.normals((args.nvec, p), 1), device=dev)
        X = torch.empty_like(B)
        ctx.solve(emb, B, rtol=1e-30, maxit=args.cg_iters, X=X)   # warm-up
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        times = []
        for _ in range(args.reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, iters, _, _ = ctx.solve(emb, B, rtol=1e-30, maxit=args.cg_iters, X=X)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / max(1, iters))
        print(json.dumps({"workload": w.name, "nvec": args.nvec, "prec": args.prec, "schedule": tuned,
                          "cg_iters": args.cg_iters, "ms_per_iteration": float(np.mean(times)),
                          "launches": kry.launch_count()}))
        ctx.close()
        return
    V = torch.tensor(I.normals((args.nvec, p), 1), dtype=dt, device=dev)
    out = torch.empty_like(V)
    ctx.matvec(emb, V, out)                      # warm-up (allocates the slab)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.matvec(emb, V, out)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    M1 = M2 = 1
    while M1 < 2 * w.n1:
        M1 *= 2
    while M2 < 2 * w.n2:
        M2 *= 2
    bpv = 16.0 * w.n1 * M2 + 16.0 * p
    ms = float(np.mean(times))
    print(json.dumps({"workload": w.name, "nvec": args.nvec, "prec": args.prec, "schedule": tuned, "ms_per_call": ms,
                      "model_bytes_per_call": bpv * args.nvec + 4.0 * M1 * M2,
                      "model_GBps": (bpv * args.nvec + 4.0 * M1 * M2) / ms / 1e6}))
    ctx.close()


if __name__ == "__main__":
    main()
