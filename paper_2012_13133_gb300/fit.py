"""Profile-likelihood estimation of the covariance parameters (Sec. 3.4, "Optimization details").

Two objectives, both evaluated on the GPU through the C ABI (the host only forms derivatives and
steps a limited-memory quasi-Newton method, L-BFGS-B, on log-transformed positive parameters, as the
paper's log transform removes the positivity constraints):

* "marginal" (default): the marginal Gaussian log-likelihood of the hot path (SLQ log-det with fixed
  probes, CG, beta profiled by GLS; kry_profile_loglik) over log sigma^2, log tau^2 and log range,
  with central-difference gradients (the fixed probes make the objective deterministic).
* "paper": the paper's approximate profile log-likelihood (Eq. prof_lik: genHyBR with k steps and
  the BCCB log-det) over log range and beta with the variances held fixed, using the approximate
  gradient of Appendix A (Eq. approx_grad) from kry_genhybr.  Eq. prof_lik is the profile of the
  joint density of (x, y): its -n/2 log sigma^2 term grows without bound as sigma^2 -> 0 (x_hat -> 0
  keeps the other terms finite), and likewise -p/2 log tau^2 as tau^2 -> 0, so the variances are
  not estimated from it here.

The paper itself runs MATLAB's trust-region fminunc with a rank-one Hessian from the gradient.

  python -m paper_2012_13133_gb300.fit --workload grid1024
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


def _log_bounds(ctx, variances):
    """Box on the log parameters: variances in [1e-6, 1e4], range from half a cell to 2."""
    cell = 1.0 / max(ctx.n1, ctx.n2)
    var = [(math.log(1e-6), math.log(1e4))] * variances
    return var + [(math.log(0.5 * cell), math.log(2.0))]


def marginal_objective(ctx, y, X, cov0, opts, h=None):
    """(f, counter) with f(v) = (-loglik, -gradient) at v = [log sigma^2, log tau^2, log range]: the
    marginal log-likelihood of kry_profile_loglik (beta profiled by GLS; nu and anisotropy from cov0)
    and its central differences with step h (default 1e-4 for FP64 vectors, 1e-2 for FP32, whose
    rounding noise in the log-likelihood would swamp a smaller step).  A setting where the solve
    breaks down (KryError) scores below every value seen so far, so a line search backs off from it."""
    from paper_2012_13133_gb300 import kry

    if h is None:
        h = 1e-4 if opts.prec == kry.KRY_F64 else 1e-2
    evals = [0]
    worst = [None]

    def cov_of(v):
        return I.Cov(math.exp(v[0]), math.exp(v[2]), cov0.nu, math.exp(v[1]), angle=cov0.angle, ratio=cov0.ratio)

    def ll(v):
        evals[0] += 1
        try:
            f = float(ctx.profile_loglik(y, X, [cov_of(v)], opts)["loglik"][0])
        except kry.KryError:
            return worst[0] - 1e3 * (1.0 + abs(worst[0])) if worst[0] is not None else -1e300
        worst[0] = f if worst[0] is None else min(worst[0], f)
        return f

    def f(v):
        v = np.asarray(v, dtype=np.float64)
        val = ll(v)
        g = np.empty(3)
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            g[j] = (ll(v + e) - ll(v - e)) / (2 * h)
        return -val, -g

    f.cov_of = cov_of
    return f, evals


def fit_marginal(ctx, y, X, cov0, opts, maxiter=100, h=None):
    """Maximise the marginal log-likelihood (kry_profile_loglik) over log sigma^2, log tau^2 and log
    range (nu and anisotropy fixed; beta profiled by GLS).  y: (p,) float64 CUDA; X: (ncov, p) float64
    CUDA; opts: kry.Opts (its probes and seed stay fixed); h as in marginal_objective.  Returns
    dict(cov, beta, loglik, evaluations, converged, message)."""
    import scipy.optimize

    f, evals = marginal_objective(ctx, y, X, cov0, opts, h)
    v0 = np.array([math.log(cov0.sigma2), math.log(cov0.tau2), math.log(cov0.range)])
    res = scipy.optimize.minimize(f, v0, jac=True, method="L-BFGS-B", bounds=_log_bounds(ctx, 2),
                                  options=dict(maxiter=maxiter))
    cov = f.cov_of(res.x)
    final = ctx.profile_loglik(y, X, [cov], opts)
    return dict(cov=cov, beta=np.asarray(final["beta"][0]), loglik=float(final["loglik"][0]),
                evaluations=evals[0] + 1, converged=bool(res.success), message=str(res.message))


def paper_objective(ctx, y, X, cov0, k):
    """(f, counter) with f(v) = (-pl, -gradient) at v = [log range, beta...]: the paper's approximate
    profile log-likelihood (Eq. prof_lik) from kry_genhybr with k steps, sigma^2 and tau^2 held at
    cov0's values.  The gradient is the approximate one of Appendix A (Eq. approx_grad) by the chain
    rule: d/d log range = range * d/d range, and d/d beta = lambda_e^2 X^T psi_k* (b = y - X beta
    enters pl only through psi_k* = b - A x_k*)."""
    Xh = X.double()
    evals = [0]

    def cov_of(v):
        return I.Cov(cov0.sigma2, math.exp(v[0]), cov0.nu, cov0.tau2, angle=cov0.angle, ratio=cov0.ratio)

    def f(v):
        import torch

        v = np.asarray(v, dtype=np.float64)
        cov, beta = cov_of(v), v[1:]
        b = (y - Xh.T @ torch.tensor(beta, dtype=torch.float64, device=y.device)).contiguous()
        g = ctx.genhybr(cov, b, k, want_x=False, gradient=True)
        evals[0] += 1
        d = np.empty(v.size)
        d[0] = cov.range * g["grad"][1]
        d[1:] = (1.0 / cov.tau2) * (Xh @ g["psi"]).cpu().numpy()
        return -g["pl"], -d

    f.cov_of = cov_of
    return f, evals


def fit_paper(ctx, y, X, cov0, beta0, k=50, maxiter=200):
    """Maximise the paper's approximate profile log-likelihood (Eq. prof_lik) over log range and beta
    with sigma^2 and tau^2 held at cov0's values, using the gradient of Eq. approx_grad
    (paper_objective).  y: (p,) float64 CUDA; X: (ncov, p) float64 CUDA.  Returns dict(cov, beta, pl,
    evaluations, converged, message)."""
    import scipy.optimize

    f, evals = paper_objective(ctx, y, X, cov0, k)
    v0 = np.concatenate([[math.log(cov0.range)], np.asarray(beta0, dtype=np.float64)])
    bounds = _log_bounds(ctx, 0) + [(None, None)] * (v0.size - 1)
    res = scipy.optimize.minimize(f, v0, jac=True, method="L-BFGS-B", bounds=bounds,
                                  options=dict(maxiter=maxiter, ftol=1e-13, gtol=1e-7))
    return dict(cov=f.cov_of(res.x), beta=np.asarray(res.x[1:]), pl=-float(res.fun), evaluations=evals[0],
                converged=bool(res.success), message=str(res.message))


def main():
    import torch

    from paper_2012_13133_gb300 import kry

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="grid1024", choices=["grid1024", "search512", "tiny32"])
    ap.add_argument("--k", type=int, default=50, help="genGK steps (objective 'paper')")
    ap.add_argument("--objective", default="marginal", choices=["marginal", "paper"])
    args = ap.parse_args()
    w = I.WORKLOADS[args.workload]
    dev = torch.device("cuda:0")
    ctx = kry.Context(0)
    mask = I.make_mask(w)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(dev))
    S1, S2 = I.cell_centres(w.n1, w.n2)
    X = I.covariates(S1[mask], S2[mask])
    M1, M2, _ = ctx.sample_size(w.cov)
    xi, eps = I.data_noise(M1, M2, p, w.data_seed)
    field = ctx.sample(w.cov, M1, M2, torch.tensor(xi, device=dev)).cpu().numpy()
    y = X @ np.array(w.beta) + field[mask] + math.sqrt(w.cov.tau2) * eps
    yt, Xt = torch.tensor(y, device=dev), torch.tensor(X.T.copy(), device=dev)
    # start: variances and range off by 2x (the paper objective holds the variances at the truth)
    if args.objective == "paper":
        start = I.Cov(w.cov.sigma2, 2.0 * w.cov.range, w.cov.nu, w.cov.tau2, w.cov.angle, w.cov.ratio)
    else:
        start = I.Cov(2.0 * w.cov.sigma2, 2.0 * w.cov.range, w.cov.nu, 2.0 * w.cov.tau2, w.cov.angle, w.cov.ratio)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.objective == "paper":
        res = fit_paper(ctx, yt, Xt, start, np.zeros(X.shape[1]), k=args.k)
    else:
        # FP32 where it resolves K, FP64 for settings the trajectory reaches that it does not
        opts = kry.Opts(prec=kry.KRY_AUTO, nprobe=16, nsteps=40, seed=w.probe_seed, rtol=1e-8, maxit=20000,
                        reorth=1)
        res = fit_marginal(ctx, yt, Xt, start, opts)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    ctx.close()
    c = res["cov"]
    print(json.dumps({"workload": w.name, "objective": args.objective, "k": args.k, "seconds": t,
                      "evaluations": res["evaluations"], "converged": res["converged"],
                      "value": res.get("loglik", res.get("pl")),
                      "estimate": {"sigma2": c.sigma2, "tau2": c.tau2, "range": c.range,
                                   "beta": res["beta"].tolist()},
                      "truth": {"sigma2": w.cov.sigma2, "tau2": w.cov.tau2, "range": w.cov.range,
                                "beta": list(w.beta)},
                      "start": {"sigma2": start.sigma2, "tau2": start.tau2, "range": start.range}}))


if __name__ == "__main__":
    main()
