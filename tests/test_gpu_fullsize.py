"""Parity at the benchmark's full size (grid1024: 1024 x 1024 grid, 50% observed,
Matern 3/2, range 0.05, nugget 0.05) in the launch configuration bench.py
times: 64 probes x 60 Lanczos steps in one batch with partial
reorthogonalisation, FP32 CG on the four right-hand sides [y, X] to a true
relative residual of 1e-6, GLS, and the kriging mean at all 524,288
unobserved cells.

The data are the oracle's: y = X beta + x + tau eps with x drawn by the
oracle's circulant-embedding sampler from the seeded white noise.  The
expected values come from tests/golden/grid1024_oracle.npz, written by
tests/golden/make_fullsize.py, which calls only the FP64 oracle: the 64
per-probe quadrature values with the same probes and a fully
reorthogonalised basis (the exact Gauss rule), CG to 1e-10, the GLS beta, the
log-likelihood and every kriging mean.

Tolerances (stated in the test): per-probe values, log det and loglik 1e-3
relative (the log-det tolerance at the stated probe and step counts); the
kriging means 1e-4 relative l2 over all targets; beta 1e-4 relative l2."""
import math
import os

import numpy as np
import pytest

from oracle import kryoracle as O
from paper_2012_13133_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2012_13133_gb300 import kry  # noqa: E402

DEV = torch.device("cuda:0")
W = I.WORKLOADS["grid1024"]
GOLD = os.path.join(os.path.dirname(__file__), "golden", "grid1024_oracle.npz")

TOL_LOGDET = 1e-3
TOL_MEAN = 1e-4
TOL_BETA = 1e-4


def oracle_data(w):
    """The golden script's data recipe (oracle sampler on its PSD torus)."""
    from tests.golden.make_fullsize import oracle_data as od
    return od(w)


@pytest.fixture(scope="module")
def problem():
    gold = dict(np.load(GOLD))
    mask, X, y, M1, M2 = oracle_data(W)
    assert (M1, M2) == tuple(gold["sample_M"])
    assert float(y.sum()) == pytest.approx(float(gold["y_sum"]), rel=1e-9, abs=1e-6)
    assert float(np.linalg.norm(y)) == pytest.approx(float(gold["y_norm"]), rel=1e-12)
    ctx = kry.Context(0)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    assert p == int(gold["p"])
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y, gold=gold)
    ctx.close()


def _opts():
    return kry.Opts(prec=kry.KRY_F32, nprobe=W.nprobe, nsteps=W.nsteps, seed=W.probe_seed, rtol=W.cg_tol,
                    maxit=20000, reorth=W.reorth)


def test_loglik_and_kriging_means_match_oracle_at_full_size(problem):
    ctx, y, X, mask, gold = problem["ctx"], problem["y"], problem["X"], problem["mask"], problem["gold"]
    emb = ctx.embed(W.cov, kry.KRY_F32)
    ctx.autotune(emb, W.nprobe)
    ctx.autotune(emb, X.shape[1] + 1)
    emb.free()
    cells = np.flatnonzero(~mask.ravel()).astype(np.int64)
    S1, S2 = I.cell_centres(W.n1, W.n2)
    Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
    res = ctx.loglik_krige(W.cov, _opts(), torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV),
                           cells=torch.tensor(cells, device=DEV), Xc=torch.tensor(Xc.T.copy(), device=DEV))
    assert res["status"] == kry.KRY_OK
    ld_err = abs(res["logdet"] - float(gold["logdet"])) / abs(float(gold["logdet"]))
    ll_err = abs(res["loglik"] - float(gold["loglik"])) / abs(float(gold["loglik"]))
    beta_err = np.linalg.norm(res["beta"] - gold["beta"]) / np.linalg.norm(gold["beta"])
    mc = res["mean_cells"].cpu().numpy()
    ref = gold["means"].astype(np.float64)
    mean_err = np.linalg.norm(mc - ref) / np.linalg.norm(ref)
    print(f"grid1024 vs oracle: logdet {ld_err:.2e}, loglik {ll_err:.2e}, beta {beta_err:.2e}, means {mean_err:.2e}")
    assert ld_err <= TOL_LOGDET
    assert ll_err <= TOL_LOGDET
    assert beta_err <= TOL_BETA
    assert mc.shape == ref.shape and mean_err <= TOL_MEAN


def test_every_probe_matches_oracle_at_full_size(problem):
    ctx, gold = problem["ctx"], problem["gold"]
    emb = ctx.embed(W.cov, kry.KRY_F32)
    ctx.autotune(emb, W.nprobe)
    ld, se, per = ctx.logdet(emb, W.nprobe, W.nsteps, W.probe_seed, reorth=W.reorth)
    emb.free()
    ref = gold["per_probe"]
    assert per.shape == ref.shape == (W.nprobe,)
    err = np.abs(per - ref) / np.abs(ref)
    print(f"grid1024 per-probe quadrature vs oracle: max {err.max():.2e}, median {np.median(err):.2e}")
    assert err.max() <= TOL_LOGDET
    assert ld == pytest.approx(float(gold["logdet"]), rel=TOL_LOGDET)


def test_solve_meets_its_residual_at_full_size(problem):
    ctx = problem["ctx"]
    emb32 = ctx.embed(W.cov, kry.KRY_F32)
    B = np.vstack([problem["y"], problem["X"].T])
    Bt = torch.tensor(B, device=DEV)
    Xs, iters, relres, st = ctx.solve(emb32, Bt, rtol=W.cg_tol, maxit=20000)
    assert st == kry.KRY_OK and relres <= W.cg_tol
    emb64 = ctx.embed(W.cov, kry.KRY_F64)
    KX = ctx.matvec(emb64, Xs.contiguous())
    for k in range(B.shape[0]):
        r = float(torch.linalg.norm(Bt[k] - KX[k]) / torch.linalg.norm(Bt[k]))
        assert r <= W.cg_tol * 1.0001, (k, r)
    emb32.free()
    emb64.free()


def test_bccb_logdet_at_full_size(problem):
    """BCCB log-det and range derivative of the grid1024 covariance (2048^2 torus) vs the oracle."""
    ld, dl = problem["ctx"].bccb_logdet(W.cov)
    ref_ld, ref_dl = O.bccb_logdet(W.n1, W.n2, W.cov, "scaled")
    assert ld == pytest.approx(ref_ld, rel=1e-9)
    assert dl == pytest.approx(ref_dl, rel=1e-7)
