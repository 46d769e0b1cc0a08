"""Write the FP64 oracle's expected values for the full-size workloads.

Calls only ``oracle/`` and the seeded input recipes of
``paper_2012_13133_gb300.inputs``; nothing here touches the CUDA library.  The
GPU parity tests (tests/test_gpu_fullsize.py, tests/test_gpu_workloads.py)
rebuild the same data with the oracle's own sampler and compare the library's
results with the files written here.

What the oracle computes, per workload (all FP64, the paper's definitions):

* data y = X beta + x + tau eps, x the circulant-embedding sample of the
  seeded white noise on the oracle's PSD torus (Sec. 3.5 sampler, Eq. obs_mod);
* the per-probe stochastic Lanczos quadrature values of log det K with the
  workload's Rademacher probes and step count, with the Lanczos basis fully
  reorthogonalised (the exact Gauss rule; stochastic trace alternative of
  Sec. 3.3);
* K^-1 [y, X] by CG to a relative residual of ``--tol`` (Sec. 3; with
  ``--precond`` preconditioned by the torus inverse, which reaches the same
  solution in far fewer iterations on clustered gaps), the GLS beta and the
  marginal log-likelihood;
* kriging means X_t beta + sigma^2 Sigma_{t,o} w, w = K^-1 (y - X beta)
  (Eq. act_xhat plus the trend), at every unobserved cell (grid1024) or at a
  seeded sample of them (large4096).

For large4096 the per-probe values may be restricted to the first ``--probes``
probes (``probe_ids`` in the file; log det and log-likelihood then use those
probes), since each fully reorthogonalised 80-step basis at 4096^2 takes about
20 GB of host memory per worker.  ``--ckpt DIR`` keeps the CG solution there
and reuses it when the script runs again.

Usage (from the repository root; hours for large4096 on a few cores):
    python tests/golden/make_fullsize.py grid1024  [--procs 4] [--threads 2]
    python tests/golden/make_fullsize.py search512 [--procs 4] [--threads 2]
    python tests/golden/make_fullsize.py large4096 --tol 1e-8 --precond --probes 8 \
        [--procs 4] [--threads 1] [--slq-procs 2] [--slq-threads 3] [--ckpt DIR]
"""
from __future__ import annotations

import argparse
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLD = os.path.dirname(os.path.abspath(__file__))

# seeded choice of the large4096 cells whose kriging means are stored
LARGE_SAMPLE_SEED = 21
LARGE_SAMPLE_CELLS = 2048
# search512 settings (indices into the 8 ranges x 4 smoothness grid, range-major) stored:
# the easiest (range 0.02, nu 0.5), two in between and the hardest (range 0.16, nu 2.5)
SEARCH_SETTINGS = (0, 9, 22, 31)


def oracle_data(w, cov=None):
    """(mask, X, y, M1, M2) of workload w with the oracle's sampler: the white noise of
    inputs.data_noise on the smallest torus whose embedding is PSD (O.sample_embed_size)."""
    from oracle import kryoracle as O
    from paper_2012_13133_gb300 import inputs as I
    mask = I.make_mask(w)
    p = int(mask.sum())
    M1, M2 = O.sample_embed_size(w.n1, w.n2, w.cov)
    xi, eps = I.data_noise(M1, M2, p, w.data_seed)
    y, X, _ = O.make_data(w.n1, w.n2, mask, w.cov, w.beta, xi, eps)
    return mask, X, y, M1, M2


def search_settings(w):
    from paper_2012_13133_gb300 import inputs as I
    return [I.Cov(1.0, r, nu, w.cov.tau2) for r in w.extra["ranges"] for nu in w.extra["nus"]]


# ---------------------------------------------------------------- pool workers

_P = None


def _init(name, threads, cov_index):
    """Worker set-up: the oracle's FFT thread count and its own copy of the problem."""
    global _P
    from oracle import kryoracle as O
    from paper_2012_13133_gb300 import inputs as I
    O._WORKERS = threads
    w = I.WORKLOADS[name]
    cov = w.cov if cov_index < 0 else search_settings(w)[cov_index]
    _P = O.FFTProblem(w.n1, w.n2, I.make_mask(w), cov)


def _probe(args):
    """Quadrature value of one probe (full reorthogonalisation)."""
    k, nsteps, seed = args
    from oracle import kryoracle as O
    z = O.rademacher_probe(seed, k, _P.p)
    a, b = O.lanczos(_P.matvec, z, nsteps, reorth=True)
    return k, O.gauss_quadrature_logdet(a, b, float(z @ z)), len(a)


def _cg(args):
    """CG solve of one right-hand side (preconditioned by the torus inverse if asked: the same
    solution in fewer iterations)."""
    j, b, tol, precond = args
    x, it = _P.solve(b, tol, precond=precond)
    return j, x, it


def run_problem(name, cov_index, y, X, tol, procs, threads, log, precond=False, nprobe=None, slq_procs=None,
                slq_threads=None, ckpt=None):
    """Per-probe SLQ values (probes 0 .. nprobe-1, all by default), the CG solve of [y, X], GLS
    beta and loglik for one setting.  ckpt: file that keeps the CG solution between runs."""
    from oracle import kryoracle as O
    from paper_2012_13133_gb300 import inputs as I
    w = I.WORKLOADS[name]
    ctx = mp.get_context("spawn")
    t0 = time.time()
    B = np.column_stack([y, X])
    if ckpt and os.path.exists(ckpt):
        c = np.load(ckpt)
        Z, iters = c["Z"], [int(i) for i in c["iters"]]
        assert Z.shape == B.shape
        log(f"  CG solution from {ckpt}")
    else:
        with ctx.Pool(min(procs, B.shape[1]), initializer=_init, initargs=(name, threads, cov_index)) as pool:
            sols = sorted(pool.map(_cg, [(j, B[:, j], tol, precond) for j in range(B.shape[1])]),
                          key=lambda r: r[0])
        Z = np.stack([s[1] for s in sols], axis=1)
        iters = [s[2] for s in sols]
        if ckpt:
            np.savez(ckpt, Z=Z, iters=np.array(iters))
    log(f"  CG {iters} iterations, {time.time() - t0:.0f} s")
    t0 = time.time()
    nprobe = w.nprobe if nprobe is None else nprobe
    with ctx.Pool(slq_procs or procs, initializer=_init, initargs=(name, slq_threads or threads, cov_index)) as pool:
        res = sorted(pool.map(_probe, [(k, w.nsteps, w.probe_seed) for k in range(nprobe)], chunksize=1),
                     key=lambda r: r[0])
    per = np.array([r[1] for r in res])
    steps = np.array([r[2] for r in res])
    log(f"  SLQ {nprobe} probes, {time.time() - t0:.0f} s")
    ld = float(per.mean())
    se = float(per.std(ddof=1) / math.sqrt(per.size))
    ll, beta, quad = O.gls_loglik(ld, Z[:, 0], Z[:, 1:], y, X)
    return dict(per_probe=per, probe_ids=np.arange(nprobe), lanczos_steps=steps, logdet=ld, logdet_se=se, loglik=ll,
                beta=beta, quad=quad, cg_iters=np.array(iters), Z=Z)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["grid1024", "search512", "large4096"])
    ap.add_argument("--procs", type=int, default=4)
    ap.add_argument("--threads", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--precond", action="store_true",
                    help="CG preconditioned by the torus inverse (same solution, fewer iterations)")
    ap.add_argument("--probes", type=int, default=None, help="per-probe values for the first K probes only")
    ap.add_argument("--slq-procs", type=int, default=None)
    ap.add_argument("--slq-threads", type=int, default=None)
    ap.add_argument("--ckpt", default=None, help="directory that keeps the CG solution between runs")
    args = ap.parse_args()

    from oracle import kryoracle as O
    from paper_2012_13133_gb300 import inputs as I
    O._WORKERS = args.procs * args.threads
    w = I.WORKLOADS[args.workload]
    t_start = time.time()

    def log(msg):
        print(f"[{time.time() - t_start:7.0f} s] {msg}", flush=True)

    mask, X, y, M1, M2 = oracle_data(w)
    log(f"{w.name}: p = {y.size}, sampling torus {M1} x {M2}")
    out = dict(tol=args.tol, precond=int(args.precond), sample_M=np.array([M1, M2]), y_sum=float(y.sum()),
               y_norm=float(np.linalg.norm(y)), p=y.size)
    S1, S2 = I.cell_centres(w.n1, w.n2)

    if w.name in ("grid1024", "large4096"):
        ck = os.path.join(args.ckpt, f"{w.name}_cg_{args.tol:g}.npz") if args.ckpt else None
        r = run_problem(w.name, -1, y, X, args.tol, args.procs, args.threads, log, args.precond, args.probes,
                        args.slq_procs, args.slq_threads, ck)
        Z = r.pop("Z")
        out.update(r)
        wts = Z[:, 0] - Z[:, 1:] @ r["beta"]
        miss = np.flatnonzero(~mask.ravel())
        if w.name == "grid1024":
            cells = miss
        else:
            pick = np.sort(np.random.default_rng(LARGE_SAMPLE_SEED).choice(miss.size, LARGE_SAMPLE_CELLS,
                                                                             replace=False))
            cells = miss[pick]
            out["cells"] = cells
        P = O.FFTProblem(w.n1, w.n2, mask, w.cov)
        Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
        means = Xc @ r["beta"] + P.sigma_at(wts, cells)
        out["means"] = means.astype(np.float32) if w.name == "grid1024" else means
        log(f"  means at {cells.size} cells")
    else:
        thetas = search_settings(w)
        out["settings"] = np.array(SEARCH_SETTINGS)
        per, ll, ld, beta, its = [], [], [], [], []
        for t in SEARCH_SETTINGS:
            log(f"setting {t}: range {thetas[t].range:g}, nu {thetas[t].nu:g}")
            r = run_problem(w.name, t, y, X, args.tol, args.procs, args.threads, log)
            per.append(r["per_probe"])
            ll.append(r["loglik"])
            ld.append(r["logdet"])
            beta.append(r["beta"])
            its.append(r["cg_iters"])
        out.update(per_probe=np.array(per), loglik=np.array(ll), logdet=np.array(ld), beta=np.array(beta),
                   cg_iters=np.array(its))
    path = os.path.join(GOLD, f"{w.name}_oracle.npz")
    np.savez_compressed(path, **out)
    log(f"wrote {path}")


if __name__ == "__main__":
    main()
