"""Parity at the full sizes of the two workloads that the benchmark does not time.

search512 (512 x 512 grid, 70% observed, data from Matern nu = 1, range 0.08):
the batched profile-likelihood search over 32 covariance settings (ranges
0.02..0.16 x nu in {0.5, 1, 1.5, 2.5}, sigma^2 = 1, tau^2 = 0.1) with 32 probes
x 50 Lanczos steps per setting in shared launches.  Checked: the
log-likelihoods, log-determinants and every probe's quadrature value at four
settings (the easiest, two in between, the hardest) against the FP64 oracle;
batched equals single calls; the hardest setting's solve meets its true FP64
residual.

large4096 (4096 x 4096 grid, ~30% missing in circular gaps, anisotropic
exponential covariance) in its launch configuration: 32 probes x 80 steps with
partial reorthogonalisation, CG on [y, X] to 1e-6, kriging means at every
missing cell.  Checked against the oracle: the log-likelihood, log det, beta,
the quadrature values of the probes the oracle stores (the first 8; each fully
reorthogonalised 80-step basis at this size takes ~20 GB of host memory), and
the kriging means at 2048 seeded missing cells (the oracle's own CG weights);
K v entries from dense covariance rows.

The data of both are the oracle's (its circulant-embedding sampler on the
seeded white noise).  Expected values: tests/golden/{search512,
large4096}_oracle.npz, written by tests/golden/make_fullsize.py from the
oracle alone.  Tolerances: log det, loglik and per-probe values 1e-3
relative; kriging means 1e-4 relative l2; beta 1e-4 relative l2.
"""
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
W3 = I.WORKLOADS["search512"]
W5 = I.WORKLOADS["large4096"]
GOLD = os.path.join(os.path.dirname(__file__), "golden")

TOL_LOGDET = 1e-3
TOL_MEAN = 1e-4
TOL_BETA = 1e-4


def load_gold(w):
    return dict(np.load(os.path.join(GOLD, f"{w.name}_oracle.npz")))


def make_problem(ctx, w, gold):
    """Mask, p, X and y of workload w with the oracle's sampler (the golden script's recipe), checked
    against the data summary stored with the expected values."""
    from tests.golden.make_fullsize import oracle_data
    mask, X, y, M1, M2 = oracle_data(w)
    assert (M1, M2) == tuple(gold["sample_M"])
    assert float(np.linalg.norm(y)) == pytest.approx(float(gold["y_norm"]), rel=1e-12)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    assert p == int(gold["p"]) == y.size
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


def rel(a, b):
    return abs(a - b) / abs(b)


# ---------------------------------------------------------------------------------- search512

def search_thetas():
    return [I.Cov(1.0, r, nu, W3.cov.tau2) for r in W3.extra["ranges"] for nu in W3.extra["nus"]]


@pytest.fixture(scope="module")
def search():
    gold = load_gold(W3)
    ctx = kry.Context(0)
    mask, p, X, y = make_problem(ctx, W3, gold)
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y, gold=gold)
    ctx.close()


def _search_opts():
    return kry.Opts(prec=kry.KRY_F32, nprobe=W3.nprobe, nsteps=W3.nsteps, seed=W3.probe_seed, rtol=W3.cg_tol,
                    maxit=30000, reorth=W3.reorth)


def test_search512_batched_settings_match_oracle(search):
    ctx, X, y, gold = search["ctx"], search["X"], search["y"], search["gold"]
    thetas = search_thetas()
    assert len(thetas) == 32
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    batch = ctx.profile_loglik(yt, Xt, thetas, _search_opts())
    assert batch["status"] == kry.KRY_OK
    assert np.all(np.isfinite(batch["loglik"]))
    for j, t in enumerate(gold["settings"]):
        e_ll = rel(batch["loglik"][t], gold["loglik"][j])
        e_ld = rel(batch["logdet"][t], gold["logdet"][j])
        e_b = np.linalg.norm(batch["beta"][t] - gold["beta"][j]) / np.linalg.norm(gold["beta"][j])
        print(f"search512 setting {t}: loglik {e_ll:.2e}, logdet {e_ld:.2e}, beta {e_b:.2e}")
        assert e_ll <= TOL_LOGDET and e_ld <= TOL_LOGDET, (t, e_ll, e_ld)
        assert e_b <= TOL_BETA, (t, e_b)


def test_search512_every_probe_matches_oracle(search):
    ctx, gold = search["ctx"], search["gold"]
    thetas = search_thetas()
    for j, t in enumerate(gold["settings"]):
        emb = ctx.embed(thetas[t], kry.KRY_F32)
        _, _, per = ctx.logdet(emb, W3.nprobe, W3.nsteps, W3.probe_seed, reorth=W3.reorth)
        emb.free()
        err = np.abs(per - gold["per_probe"][j]) / np.abs(gold["per_probe"][j])
        print(f"search512 setting {t}: per-probe max {err.max():.2e}")
        assert err.max() <= TOL_LOGDET, (t, err.max())


def test_search512_batched_settings_equal_single_calls(search):
    ctx, X, y = search["ctx"], search["X"], search["y"]
    thetas = search_thetas()
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    batch = ctx.profile_loglik(yt, Xt, thetas, _search_opts())
    for t in (0, len(thetas) - 1):
        one = ctx.profile_loglik(yt, Xt, [thetas[t]], _search_opts())
        assert batch["loglik"][t] == pytest.approx(one["loglik"][0], rel=1e-6)
        assert batch["logdet"][t] == pytest.approx(one["logdet"][0], rel=1e-6)


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
    gold = load_gold(W5)
    ctx = kry.Context(0)
    mask, p, X, y = make_problem(ctx, W5, gold)
    sites = O.observed_sites(W5.n1, W5.n2, mask)
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y, sites=sites, gold=gold)
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


def test_large4096_loglik_krige_match_oracle(large):
    ctx, X, y, mask, gold = large["ctx"], large["X"], large["y"], large["mask"], large["gold"]
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    opts = kry.Opts(prec=kry.KRY_F32, nprobe=W5.nprobe, nsteps=W5.nsteps, seed=W5.probe_seed, rtol=W5.cg_tol,
                    maxit=60000, reorth=W5.reorth)
    cells = np.flatnonzero(~mask.ravel()).astype(np.int64)
    S1, S2 = I.cell_centres(W5.n1, W5.n2)
    Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
    res = ctx.loglik_krige(W5.cov, opts, yt, Xt, cells=torch.tensor(cells, device=DEV),
                           Xc=torch.tensor(Xc.T.copy(), device=DEV))
    assert res["status"] == kry.KRY_OK
    # the oracle's log det and log-likelihood average the probes it stores (probe_ids, the
    # first K of the workload's probes): the library's log-likelihood is compared with its own
    # log det replaced by the mean of its values on those probes (l + logdet / 2 does not
    # depend on the probes)
    ids = gold["probe_ids"] if "probe_ids" in gold else np.arange(W5.nprobe)
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    _, _, per = ctx.logdet(emb, W5.nprobe, W5.nsteps, W5.probe_seed, reorth=W5.reorth)
    emb.free()
    assert float(per.mean()) == pytest.approx(res["logdet"], rel=1e-12)
    ld_sub = float(per[ids].mean())
    e_ll = rel(res["loglik"] + 0.5 * res["logdet"] - 0.5 * ld_sub, float(gold["loglik"]))
    e_ld = rel(ld_sub, float(gold["logdet"]))
    e_b = np.linalg.norm(res["beta"] - gold["beta"]) / np.linalg.norm(gold["beta"])
    # the stored cells are a seeded sample of the missing cells, in increasing order
    pos = np.searchsorted(cells, gold["cells"])
    assert np.array_equal(cells[pos], gold["cells"])
    mc = res["mean_cells"].cpu().numpy()[pos]
    e_m = np.linalg.norm(mc - gold["means"]) / np.linalg.norm(gold["means"])
    print(f"large4096 vs oracle: loglik {e_ll:.2e}, logdet {e_ld:.2e}, beta {e_b:.2e}, means {e_m:.2e}")
    assert e_ll <= TOL_LOGDET and e_ld <= TOL_LOGDET
    assert e_b <= TOL_BETA
    assert e_m <= TOL_MEAN


def test_large4096_every_probe_matches_oracle(large):
    ctx, gold = large["ctx"], large["gold"]
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    _, _, per = ctx.logdet(emb, W5.nprobe, W5.nsteps, W5.probe_seed, reorth=W5.reorth)
    emb.free()
    ids = gold["probe_ids"] if "probe_ids" in gold else np.arange(W5.nprobe)
    err = np.abs(per[ids] - gold["per_probe"]) / np.abs(gold["per_probe"])
    print(f"large4096 per-probe vs oracle ({len(ids)} probes): max {err.max():.2e}")
    assert err.max() <= TOL_LOGDET


def test_large4096_solve_meets_true_residual(large):
    ctx, X, y = large["ctx"], large["X"], large["y"]
    emb = ctx.embed(W5.cov, kry.KRY_F32)
    B = torch.tensor(np.vstack([y, X.T]), device=DEV)
    Z, _, relres, st = ctx.solve(emb, B, rtol=W5.cg_tol, maxit=60000)
    emb.free()
    assert st == kry.KRY_OK
    for k, r in enumerate(true_relres(ctx, W5.cov, B, Z)):
        assert r <= W5.cg_tol * 1.0001, (k, r)


def test_large4096_bccb_logdet_matches_oracle(large):
    """BCCB log-det and range derivative on the 8192^2 torus (anisotropic exponential)."""
    ld, dl = large["ctx"].bccb_logdet(W5.cov)
    ref_ld, ref_dl = O.bccb_logdet(W5.n1, W5.n2, W5.cov, "scaled")
    assert ld == pytest.approx(ref_ld, rel=1e-9)
    assert dl == pytest.approx(ref_dl, rel=1e-7)
