"""Parity at the full sizes of the two workloads that the benchmark does not time.

search512 (512 x 512 grid, 70% observed, data from Matern nu = 1, range 0.08):
the batched profile-likelihood search over 32 covariance settings (ranges
0.02..0.16 x nu in {0.5, 1, 1.5, 2.5}, sigma^2 = 1, tau^2 = 0.1) with 32 probes
x 50 Lanczos steps per setting in shared launches.  Checked: every setting
equals its own single-setting call; the per-probe quadrature values of two
probes at the easiest and the hardest setting equal the FP64 oracle's (full
reorthogonalisation) to 1e-3; the hardest setting's solve meets its true FP64
residual.

large4096 (4096 x 4096 grid, ~30% missing in circular gaps, anisotropic
exponential covariance): the 8192^2 oracle FFT takes seconds per matvec, so
the oracle evaluates sampled outputs one by one from dense covariance rows
(no FFT): entries of K v, of the residual b - K x and of the kriging mean; and
one probe's 80-step quadrature value.  The run itself uses the workload's
launch configuration: 32 probes x 80 steps with partial reorthogonalisation,
CG on [y, X] to 1e-6, kriging means at every missing cell.
"""
import math

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
W3 = I.WORKLOADS["search512"]
W5 = I.WORKLOADS["large4096"]


def make_problem(ctx, w):
    mask = I.make_mask(w)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    S1, S2 = I.cell_centres(w.n1, w.n2)
    X = I.covariates(S1[mask], S2[mask])
    M1, M2, _ = ctx.sample_size(w.cov)
    xi, eps = I.data_noise(M1, M2, p, w.data_seed)
    field = ctx.sample(w.cov, M1, M2, torch.tensor(xi, device=DEV)).cpu().numpy()
    y = X @ np.array(w.beta) + field[mask] + math.sqrt(w.cov.tau2) * eps
    return mask, p, X, y


def true_relres(ctx, cov, B, Xs):
    """||b - K x|| / ||b|| per column with the FP64 matvec."""
    emb64 = ctx.embed(cov, kry.KRY_F64)
    KX = ctx.matvec(emb64, Xs.contiguous())
    out = [float(torch.linalg.norm(B[k] - KX[k]) / torch.linalg.norm(B[k])) for k in range(B.shape[0])]
    emb64.free()
    return out


def dense_rows(sites, rows, cov, v):
    """(sigma^2 Sigma v)[i] for observed indices i in rows, from dense covariance rows."""
    out = np.zeros((len(rows),) + v.shape[1:])
    for a, i in enumerate(rows):
        c = O.covariance(sites[i, 0] - sites[:, 0], sites[i, 1] - sites[:, 1], cov)
        out[a] = c @ v
    return out


# ---------------------------------------------------------------------------------- search512

def search_thetas():
    return [I.Cov(1.0, r, nu, W3.cov.tau2) for r in W3.extra["ranges"] for nu in W3.extra["nus"]]


@pytest.fixture(scope="module")
def search():
    ctx = kry.Context(0)
    mask, p, X, y = make_problem(ctx, W3)
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y)
    ctx.close()


def test_search512_batched_settings_match_single_calls_and_oracle(search):
    ctx, X, y = search["ctx"], search["X"], search["y"]
    thetas = search_thetas()
    assert len(thetas) == 32
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    opts = kry.Opts(prec=kry.KRY_F32, nprobe=W3.nprobe, nsteps=W3.nsteps, seed=W3.probe_seed, rtol=W3.cg_tol,
                    maxit=30000, reorth=W3.reorth)
    batch = ctx.profile_loglik(yt, Xt, thetas, opts)
    assert batch["status"] == kry.KRY_OK
    assert np.all(np.isfinite(batch["loglik"]))
    for t in (0, len(thetas) - 1):
        one = ctx.profile_loglik(yt, Xt, [thetas[t]], opts)
        assert batch["loglik"][t] == pytest.approx(one["loglik"][0], rel=1e-6)
        assert batch["logdet"][t] == pytest.approx(one["logdet"][0], rel=1e-6)
    # sampled outputs against the oracle: two probes' quadrature values at the
    # easiest (range 0.02, nu 0.5) and the hardest (range 0.16, nu 2.5) setting
    for t in (0, len(thetas) - 1):
        emb = ctx.embed(thetas[t], kry.KRY_F32)
        _, _, per = ctx.logdet(emb, W3.nprobe, W3.nsteps, W3.probe_seed, reorth=W3.reorth)
        emb.free()
        P = O.FFTProblem(W3.n1, W3.n2, search["mask"], thetas[t])
        _, _, ref = P.logdet(W3.nprobe, W3.nsteps, W3.probe_seed, probe_ids=[0, W3.nprobe - 1], reorth=True)
        assert per[0] == pytest.approx(ref[0], rel=1e-3), (t, per[0], ref[0])
        assert per[-1] == pytest.approx(ref[1], rel=1e-3), (t, per[-1], ref[1])


def test_search512_hardest_setting_solve_meets_true_residual(search):
    ctx, X, y = search["ctx"], search["X"], search["y"]
    th = search_thetas()[-1]
    emb = ctx.embed(th, kry.KRY_F32)
    B = torch.tensor(np.vstack([y, X.T]), device=DEV)
    Xs, iters, relres, st = ctx.solve(emb, B, rtol=W3.cg_tol, maxit=30000)
    emb.free()
    assert st == kry.KRY_OK and relres <= W3.cg_tol
    for k, r in enumerate(true_relres(ctx, th, B, Xs)):
        assert r <= W3.cg_tol * 1.0001, (k, r)


# ---------------------------------------------------------------------------------- large4096

@pytest.fixture(scope="module")
def large():
    ctx = kry.Context(0)
    mask, p, X, y = make_problem(ctx, W5)
    sites = O.observed_sites(W5.n1, W5.n2, mask)
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y, sites=sites)
    ctx.close()


def test_large4096_matvec_rows_match_dense_covariance_rows(large):
    ctx, p, sites = large["ctx"], large["p"], large["sites"]
    V = I.normals((4, p), 17)
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    out = ctx.matvec(emb, torch.tensor(V, dtype=torch.float32, device=DEV)).double().cpu().numpy()
    emb.free()
    rows = np.random.default_rng(18).choice(p, 6, replace=False)
    ref = dense_rows(sites, rows, W5.cov, V.T) + W5.cov.tau2 * V[:, rows].T
    # FP32 FFT errors spread evenly over the entries: the sampled errors are
    # measured against the root-mean-square entry (the 1e-5 norm tolerance,
    # with a factor 3 for the spread of six samples)
    for k in range(4):
        rms = np.linalg.norm(out[k]) / math.sqrt(p)
        err = np.abs(out[k, rows] - ref[:, k]).max()
        assert err <= 3e-5 * rms, (k, err / rms)


def test_large4096_loglik_krige_at_full_size(large):
    ctx, p, X, y, sites, mask = large["ctx"], large["p"], large["X"], large["y"], large["sites"], large["mask"]
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    opts = kry.Opts(prec=kry.KRY_F32, nprobe=W5.nprobe, nsteps=W5.nsteps, seed=W5.probe_seed, rtol=W5.cg_tol,
                    maxit=60000, reorth=W5.reorth)
    cells = np.flatnonzero(~mask.ravel()).astype(np.int64)
    S1, S2 = I.cell_centres(W5.n1, W5.n2)
    Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
    res = ctx.loglik_krige(W5.cov, opts, yt, Xt, cells=torch.tensor(cells, device=DEV),
                           Xc=torch.tensor(Xc.T.copy(), device=DEV))
    assert res["status"] == kry.KRY_OK
    assert math.isfinite(res["loglik"]) and math.isfinite(res["logdet"])
    # the solve: true FP64 residual, and sampled residual entries from dense rows
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    B = torch.tensor(np.vstack([y, X.T]), device=DEV)
    Z, _, relres, st = ctx.solve(emb, B, rtol=W5.cg_tol, maxit=60000)
    emb.free()
    assert st == kry.KRY_OK
    for k, r in enumerate(true_relres(ctx, W5.cov, B, Z)):
        assert r <= W5.cg_tol * 1.0001, (k, r)
    Z = Z.cpu().numpy()
    rows = np.random.default_rng(19).choice(p, 4, replace=False)
    Bn = np.vstack([y, X.T])
    resid = Bn[:, rows].T - dense_rows(sites, rows, W5.cov, Z.T) - W5.cov.tau2 * Z[:, rows].T
    for k in range(Bn.shape[0]):
        assert np.abs(resid[:, k]).max() <= 3 * W5.cg_tol * np.linalg.norm(Bn[k]) / math.sqrt(p) * 10
    # GLS beta of that solve equals the one loglik_krige used
    A = X.T @ Z[1:].T
    g = 0.5 * (X.T @ Z[0] + Z[1:] @ y)
    beta = np.linalg.solve(0.5 * (A + A.T), g)
    assert np.allclose(res["beta"], beta, rtol=1e-5, atol=1e-7)
    # kriging means at sampled missing cells: X_t beta + sigma^2 Sigma_{t,o} K^-1 (y - X beta)
    w = Z[0] - Z[1:].T @ beta
    S = np.stack([S1.ravel(), S2.ravel()], axis=1)
    pick = np.random.default_rng(20).choice(cells.size, 4, replace=False)
    mc = res["mean_cells"].cpu().numpy()
    rms = np.linalg.norm(mc) / math.sqrt(mc.size)
    for a in pick:
        t = S[cells[a]]
        c = O.covariance(t[0] - sites[:, 0], t[1] - sites[:, 1], W5.cov)
        ref = Xc[a] @ beta + c @ w
        assert abs(mc[a] - ref) <= 1e-4 * rms, (a, mc[a], ref)


def test_large4096_probe_quadrature_matches_oracle(large):
    ctx = large["ctx"]
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    _, _, per = ctx.logdet(emb, W5.nprobe, W5.nsteps, W5.probe_seed, reorth=W5.reorth)
    emb.free()
    assert np.all(np.isfinite(per))
    P = O.FFTProblem(W5.n1, W5.n2, large["mask"], W5.cov)
    _, _, ref = P.logdet(W5.nprobe, W5.nsteps, W5.probe_seed, probe_ids=[0], reorth=True)
    assert per[0] == pytest.approx(ref[0], rel=1e-3)


def test_large4096_bccb_logdet_matches_oracle(large):
    """BCCB log-det and range derivative on the 8192^2 torus (anisotropic exponential)."""
    ld, dl = large["ctx"].bccb_logdet(W5.cov)
    ref_ld, ref_dl = O.bccb_logdet(W5.n1, W5.n2, W5.cov, "scaled")
    assert ld == pytest.approx(ref_ld, rel=1e-9)
    assert dl == pytest.approx(ref_dl, rel=1e-7)
