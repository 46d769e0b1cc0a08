"""Serving driver: a Poisson stream of likelihood and kriging requests through
the library's continuous-batching server (kry_server_*).

Requests follow the serving workload: square grids with sides drawn
log-uniformly, masks with 10-90% missing cells (half in circular gaps like
cloud cover, half uniform), Matern nu in {1/2, 3/2}, random range and nugget,
and GP data drawn by the library's circulant-embedding sampler.  The stream
is replayed against a one-slot server (one request at a time) and against a
multi-slot server: saturated (every request queued at once: the capacity of
each form) and at Poisson arrivals of a given multiple of the one-slot
throughput; each reports p50/p99 latency and requests/s.

  python -m paper_2012_13133_gb300.serve --n-requests 200 --slots 8
  python -m paper_2012_13133_gb300.serve --n-requests 2000 --precond 1 --rates 0.5,1,2 --sweep-requests 500
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2012_13133_gb300 import inputs as I  # noqa: E402


def _mask_of(sp):
    return I.mask_mixed(sp["n"], sp["n"], sp["frac_missing"], sp["mask_seed"])


def make_masks(specs, procs):
    """The request masks (host work), in a process pool started with spawn before any GPU use."""
    if procs <= 1:
        return [_mask_of(sp) for sp in specs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_mask_of, specs, chunksize=4)


def build_requests(specs, masks, device=0, nprobe=16, nsteps=50, rtol=1e-6, maxit=5000, reorth=1, precond=0):
    """Materialise request specs (inputs.serve_requests) into host arrays,
    drawing each data set with the GPU sampler."""
    import torch

    from paper_2012_13133_gb300 import kry
    ctx = kry.Context(device)
    dev = torch.device("cuda", device)
    out = []
    for sp, mask in zip(specs, masks):
        n = sp["n"]
        cov = I.Cov(1.0, sp["range"], sp["nu"], sp["tau2"])
        p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(dev))
        M1, M2, _ = ctx.sample_size(cov)
        xi, eps = I.data_noise(M1, M2, p, sp["data_seed"])
        field = ctx.sample(cov, M1, M2, torch.tensor(xi, device=dev)).cpu().numpy()
        S1, S2 = I.cell_centres(n, n)
        X = I.covariates(S1[mask], S2[mask])
        y = X @ np.array([1.0, 0.5, -0.5]) + field[mask] + math.sqrt(cov.tau2) * eps
        req = dict(spec=sp, kind=kry.KRY_REQ_LOGLIK if sp["kind"] == "loglik" else kry.KRY_REQ_KRIGE,
                   mask=mask, y=y, X=np.ascontiguousarray(X.T), cov=cov,
                   opts=kry.Opts(prec=kry.KRY_F32, nprobe=nprobe, nsteps=nsteps, seed=sp["id"], rtol=rtol,
                                 maxit=maxit, reorth=reorth, precond=precond))
        if sp["kind"] == "krige":
            cells = np.flatnonzero(~mask.ravel()).astype(np.int64)
            req["target_cells"] = cells
            req["target_X"] = np.ascontiguousarray(I.covariates(S1.ravel()[cells], S2.ravel()[cells]).T)
        out.append(req)
    ctx.close()
    return out


def replay(server, reqs, arrivals, timeout_s=3600.0):
    """Submit request i at time arrivals[i] (seconds from start); collect results.
    Returns (results in request order, wall seconds from first arrival to last completion)."""
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            delay = arrivals[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[i] = server.submit(r["kind"], r["mask"], r["y"], r["X"], r["cov"], r["opts"],
                                       r.get("target_cells"), r.get("target_X"))

    th = threading.Thread(target=submitter)
    th.start()
    results = [None] * len(reqs)
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        results[i] = server.wait(tickets[i], timeout_s)
    th.join()
    return results, time.perf_counter() - t0


def summarise(results, wall):
    lat = np.array([r["latency_ms"] for r in results])
    return {"requests": len(results), "requests_per_s": len(results) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "wall_s": wall,
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique([r["status"] for r in results],
                                                                        return_counts=True))}}


def main():
    from paper_2012_13133_gb300 import kry

    ap = argparse.ArgumentParser()
    ap.add_argument("--n-requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--rate-factor", type=float, default=1.5,
                    help="arrival rate as a multiple of the measured one-slot throughput")
    ap.add_argument("--rates", default="",
                    help="comma-separated extra rate factors replayed on the multi-slot server")
    ap.add_argument("--sweep-requests", type=int, default=0,
                    help="requests of the stream replayed at each extra rate (0: all)")
    ap.add_argument("--at-rate-requests", type=int, default=0,
                    help="requests of the stream replayed at --rate-factor on each server (0: all)")
    ap.add_argument("--side-min", type=int, default=128)
    ap.add_argument("--side-max", type=int, default=2048)
    ap.add_argument("--budget-gb", type=float, default=96.0)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--maxit", type=int, default=5000)
    ap.add_argument("--precond", type=int, default=2,
                    help="kry_opts.precond of every request (2: automatic, from the mask's interior share)")
    ap.add_argument("--mask-procs", type=int, default=8)
    args = ap.parse_args()

    w = I.WORKLOADS["serve"]
    specs = I.serve_requests(args.n_requests, args.seed, args.side_min, args.side_max, rate=1.0)
    t = time.perf_counter()

    def note(msg):
        print(f"[{time.perf_counter() - t:8.1f} s] {msg}", file=sys.stderr, flush=True)

    masks = make_masks(specs, args.mask_procs)
    note(f"{len(masks)} masks")
    reqs = build_requests(specs, masks, maxit=args.maxit, precond=args.precond)
    prep_s = time.perf_counter() - t
    note("requests built")
    budget = int(args.budget_gb * (1 << 30))
    out = {"metric": "serving p50/p99 latency and requests/s", "workload": w.name, "n_requests": len(reqs),
           "slots": args.slots, "precond": args.precond, "prep_s": prep_s}

    # capacity: every request queued at t = 0, on one slot (one request at a time) and on all slots
    one = kry.Server(0, 1, budget)
    res1, wall1 = replay(one, reqs, np.zeros(len(reqs)))
    one.close()
    out["one_slot_saturated"] = summarise(res1, wall1)
    note(f"one slot, saturated: {wall1:.1f} s")
    multi = kry.Server(0, args.slots, budget)
    resm, wallm = replay(multi, reqs, np.zeros(len(reqs)))
    multi.close()
    out[f"{args.slots}_slots_saturated"] = summarise(resm, wallm)
    note(f"{args.slots} slots, saturated: {wallm:.1f} s")
    mu1 = len(reqs) / wall1
    out["served_over_one_at_a_time"] = (len(reqs) / wallm) / mu1

    def at_rate(factor, server_slots, n):
        rate = factor * mu1
        gaps = np.random.default_rng(args.seed + 1).exponential(1.0 / rate, size=n)
        arrivals = np.cumsum(gaps) - gaps[0]
        srv = kry.Server(0, server_slots, budget)
        res, wall = replay(srv, reqs[:n], arrivals)
        srv.close()
        note(f"{server_slots} slot(s) at {factor} x: {wall:.1f} s")
        return res, dict(summarise(res, wall), rate_factor=factor, arrival_rate_per_s=rate)

    n_at = args.at_rate_requests or len(reqs)
    res_s, out["one_slot_at_rate"] = at_rate(args.rate_factor, 1, n_at)
    res_m, out[f"{args.slots}_slots_at_rate"] = at_rate(args.rate_factor, args.slots, n_at)
    sweep = []
    for f in [float(x) for x in args.rates.split(",") if x.strip()]:
        n = args.sweep_requests or len(reqs)
        sweep.append(at_rate(f, args.slots, n)[1])
    out["rate_sweep"] = sweep
    lik = [(a, b) for a, b, r in zip(res_s, res_m, reqs) if r["kind"] == kry.KRY_REQ_LOGLIK]
    out["max_rel_loglik_diff_single_vs_mixed"] = max(
        (abs(a["loglik"] - b["loglik"]) / max(1.0, abs(a["loglik"])) for a, b in lik), default=0.0)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
