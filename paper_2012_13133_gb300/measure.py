"""Timing driver for the workloads the benchmark does not time.

  python -m paper_2012_13133_gb300.measure --workload search512   # batched vs one setting at a time
  python -m paper_2012_13133_gb300.measure --workload large4096   # log-likelihood + kriging means, wall time
  python -m paper_2012_13133_gb300.measure --workload large4096 --solves   # CG on [y, X], plain vs preconditioned
  python -m paper_2012_13133_gb300.measure --workload tiny32      # FP64 evaluations per second
  python -m paper_2012_13133_gb300.measure --workload grid1024 --bccb   # BCCB log-det + derivative
  python -m paper_2012_13133_gb300.measure --workload grid1024 --bootstrap 20   # bootstrap kriging MSE
  python -m paper_2012_13133_gb300.measure --workload grid1024 --genhybr 50     # genHyBR, k = 50

Inputs are the seeded synthetic workloads of ``inputs.WORKLOADS``, resident on
the device before timing; each timed call is bracketed by device
synchronisation.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2012_13133_gb300 import inputs as I  # noqa: E402


def problem(ctx, w, dev, prec_data=None):
    import torch
    mask = I.make_mask(w)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(dev))
    S1, S2 = I.cell_centres(w.n1, w.n2)
    X = I.covariates(S1[mask], S2[mask])
    M1, M2, _ = ctx.sample_size(w.cov)
    xi, eps = I.data_noise(M1, M2, p, w.data_seed)
    field = ctx.sample(w.cov, M1, M2, torch.tensor(xi, device=dev)).cpu().numpy()
    y = X @ np.array(w.beta) + field[mask] + math.sqrt(w.cov.tau2) * eps
    return mask, p, torch.tensor(y, device=dev), torch.tensor(X.T.copy(), device=dev), S1, S2


def timed(fn):
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t


def main():
    import torch

    from paper_2012_13133_gb300 import kry

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", required=True, choices=["search512", "large4096", "tiny32", "grid1024"])
    ap.add_argument("--bccb", action="store_true", help="time the BCCB log-det and its range derivative")
    ap.add_argument("--genhybr", type=int, default=0, help="time genHyBR (Alg. 1 + Eq. prof_lik) with k steps")
    ap.add_argument("--gk-prec", default="f64", choices=["f64", "f32"], help="genHyBR vector precision")
    ap.add_argument("--gk-reorth", action="store_true", help="genHyBR with reorthogonalisation")
    ap.add_argument("--bootstrap", type=int, default=0,
                    help="time the parametric-bootstrap kriging MSE with this many replicates at all missing cells")
    ap.add_argument("--precond", type=int, default=0, help="kry_opts.precond for the CG solves (1: torus inverse)")
    ap.add_argument("--variances", type=int, default=0,
                    help="time exact simple-kriging variances at the first K of the workload's variance cells")
    ap.add_argument("--solves", action="store_true",
                    help="time CG on [y, X] with and without the torus-inverse preconditioner")
    args = ap.parse_args()
    w = I.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    ctx = kry.Context(0)
    mask, p, y, X, S1, S2 = problem(ctx, w, dev)
    out = {"workload": args.workload, "grid": [w.n1, w.n2], "p": p}
    if args.genhybr:
        b = (y - X.T @ torch.tensor(w.beta, device=dev, dtype=torch.float64)).contiguous()
        gp = kry.KRY_F32 if args.gk_prec == "f32" else kry.KRY_F64
        gr = 1 if args.gk_reorth else 0
        ctx.genhybr(w.cov, b, 2, prec=gp, reorth=gr)
        g, t = timed(lambda: ctx.genhybr(w.cov, b, args.genhybr, prec=gp, reorth=gr))
        out.update({"k": args.genhybr, "prec": args.gk_prec, "reorth": gr, "genhybr_s": t, "pl": g["pl"],
                    "z2": g["z2"], "psi2": g["psi2"]})
    elif args.variances:
        cells = I.variance_cells(w, mask)[:args.variances]
        Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
        opts = kry.Opts(prec=kry.KRY_F32, rtol=w.cg_tol, maxit=30000, precond=args.precond)
        ct, xt = torch.tensor(cells, device=dev), torch.tensor(Xc.T.copy(), device=dev)
        emb = ctx.embed(w.cov, kry.KRY_F32)
        ctx.autotune(emb, 4)
        ctx.autotune(emb, 32)
        emb.free()
        res, t = timed(lambda: ctx.krige(w.cov, opts, y, X, cells=ct, Xc=xt, variances=True))
        v = res["var_cells"].cpu().numpy()
        n_all = int(w.extra.get("n_var_cells", cells.size))
        out.update({"variance_cells": int(cells.size), "krige_with_variances_s": t, "status": int(res["status"]),
                    "precond": args.precond, "mean_var": float(v.mean()), "min_var": float(v.min()),
                    "max_var": float(v.max()), "of_cells": n_all})
    elif args.bootstrap:
        nrep = args.bootstrap
        M1, M2, _ = ctx.sample_size(w.cov)
        rng = np.random.default_rng(w.data_seed + 101)
        xi = torch.tensor(rng.standard_normal((nrep, 2, M1, M2)), device=dev)
        eps = torch.tensor(rng.standard_normal((nrep, p)), device=dev)
        cells = torch.tensor(np.flatnonzero(~mask.ravel()).astype(np.int64), device=dev)
        opts = kry.Opts(prec=kry.KRY_F32, rtol=w.cg_tol, maxit=30000, precond=args.precond)
        (var, st), t = timed(lambda: ctx.bootstrap_var(w.cov, opts, xi, eps, cells))
        v = var.cpu().numpy()
        out.update({"replicates": nrep, "cells": int(cells.numel()), "bootstrap_s": t, "status": int(st),
                    "precond": args.precond,
                    "mean_var": float(v.mean()), "min_var": float(v.min()), "max_var": float(v.max())})
    elif args.bccb:
        ctx.bccb_logdet(w.cov)
        reps = 5
        (ld, dl), t = timed(lambda: [ctx.bccb_logdet(w.cov) for _ in range(reps)][-1])
        out.update({"bccb_logdet": ld, "bccb_dlogdet_drange": dl, "ms_per_call": 1e3 * t / reps})
    elif args.workload == "grid1024":
        raise SystemExit("grid1024 is timed by bench.py; use --bccb here")
    elif args.workload == "search512":
        thetas = [I.Cov(1.0, r, nu, w.cov.tau2) for r in w.extra["ranges"] for nu in w.extra["nus"]]
        opts = kry.Opts(prec=kry.KRY_F32, nprobe=w.nprobe, nsteps=w.nsteps, seed=w.probe_seed, rtol=w.cg_tol,
                        maxit=30000, reorth=w.reorth)
        ctx.profile_loglik(y, X, thetas[:2], opts)                       # warm-up
        batch, tb = timed(lambda: ctx.profile_loglik(y, X, thetas, opts))
        singles, ts = timed(lambda: [ctx.profile_loglik(y, X, [t], opts) for t in thetas])
        # FP32 matvec work of each form (one more run of each, CUDA events per matvec)
        work = {}
        for name, fn in (("batched", lambda: ctx.profile_loglik(y, X, thetas, opts)),
                         ("one_at_a_time", lambda: [ctx.profile_loglik(y, X, [t], opts) for t in thetas])):
            ctx.profile_enable(True)
            fn()
            pr = ctx.profile_read(kry.KRY_F32)
            ctx.profile_enable(False)
            work[name] = {"matvec_calls": pr["calls"], "real_vectors": pr["vectors"], "matvec_ms": pr["ms"]}
        out["fp32_matvec_work"] = work
        # CG iterations of each setting alone (4 right-hand sides [y, X])
        B = torch.cat([y.reshape(1, -1), X], 0).contiguous()
        its = []
        for t in thetas:
            emb = ctx.embed(t, kry.KRY_F32)
            its.append(ctx.solve(emb, B, rtol=w.cg_tol, maxit=30000)[1])
            emb.free()
        out["cg_iterations_per_setting"] = its
        diff = max(abs(batch["loglik"][k] - s["loglik"][0]) / abs(s["loglik"][0]) for k, s in enumerate(singles))
        best = int(np.argmax(batch["loglik"]))
        out.update({"settings": len(thetas), "probes": w.nprobe, "lanczos_steps": w.nsteps,
                    "batched_s": tb, "one_at_a_time_s": ts, "batched_evals_per_s": len(thetas) / tb,
                    "one_at_a_time_evals_per_s": len(thetas) / ts, "max_rel_loglik_diff": diff,
                    "best_setting": {"range": thetas[best].range, "nu": thetas[best].nu},
                    "status": int(batch["status"])})
    elif args.solves:
        emb = ctx.embed(w.cov, kry.KRY_F32)
        B = torch.cat([y.reshape(1, -1), X], 0).contiguous()
        res = {}
        for pre in (False, True):
            (Z, it, rr, st), t = timed(lambda: ctx.solve(emb, B, rtol=w.cg_tol, maxit=60000, precond=pre))
            res["preconditioned" if pre else "plain"] = {"iterations": it, "relres": rr, "status": int(st),
                                                         "solve_s": t}
        emb.free()
        out.update({"rhs": int(B.shape[0]), "rtol": w.cg_tol, **res})
    elif args.workload == "large4096":
        opts = kry.Opts(prec=kry.KRY_F32, nprobe=w.nprobe, nsteps=w.nsteps, seed=w.probe_seed, rtol=w.cg_tol,
                        maxit=60000, reorth=w.reorth, precond=args.precond)
        cells = np.flatnonzero(~mask.ravel()).astype(np.int64)
        Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
        ct, xt = torch.tensor(cells, device=dev), torch.tensor(Xc.T.copy(), device=dev)
        emb = ctx.embed(w.cov, kry.KRY_F32)
        tuned = {str(nv): ctx.autotune(emb, nv) for nv in (w.nprobe, 4)}
        emb.free()
        res, t = timed(lambda: ctx.loglik_krige(w.cov, opts, y, X, cells=ct, Xc=xt))
        out.update({"probes": w.nprobe, "lanczos_steps": w.nsteps, "kriging_cells": int(cells.size),
                    "loglik_krige_s": t, "loglik": res["loglik"], "status": int(res["status"]), "precond": args.precond,
                    "tuned_schedules": tuned})
    else:
        opts = kry.Opts(prec=kry.KRY_F64, nprobe=w.nprobe, nsteps=w.nsteps, seed=w.probe_seed, rtol=w.cg_tol,
                        maxit=20000, reorth=w.reorth)
        ctx.profile_loglik(y, X, [w.cov], opts)
        n = 20
        _, t = timed(lambda: [ctx.profile_loglik(y, X, [w.cov], opts) for _ in range(n)])
        out.update({"evals_per_s": n / t, "precision": "f64"})
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
