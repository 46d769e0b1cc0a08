"""Parity at the benchmark's full size (grid1024: 1024 x 1024 grid, 50% observed,
Matern 3/2, range 0.05, nugget 0.05) in the launch configuration bench.py
times: 64 probes x 60 Lanczos steps in one batch with partial
reorthogonalisation, CG on the four right-hand sides [y, X].  The oracle
computes sampled outputs one by one (two probes' quadrature values, with full
reorthogonalisation); the solve is checked through the property that defines
it, with the FP64 matvec whose full-size parity is tested elsewhere."""
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
W = I.WORKLOADS["grid1024"]


@pytest.fixture(scope="module")
def problem():
    ctx = kry.Context(0)
    mask = I.make_mask(W)
    p = ctx.set_mask(torch.from_numpy(mask.astype(np.uint8)).to(DEV))
    S1, S2 = I.cell_centres(W.n1, W.n2)
    X = I.covariates(S1[mask], S2[mask])
    M1, M2, _ = ctx.sample_size(W.cov)
    xi, eps = I.data_noise(M1, M2, p, W.data_seed)
    field = ctx.sample(W.cov, M1, M2, torch.tensor(xi, device=DEV)).cpu().numpy()
    y = X @ np.array(W.beta) + field[mask] + math.sqrt(W.cov.tau2) * eps
    yield dict(ctx=ctx, mask=mask, p=p, X=X, y=y)
    ctx.close()


def test_logdet_probes_match_oracle_at_full_size(problem):
    ctx = problem["ctx"]
    emb = ctx.embed(W.cov, kry.KRY_F32)
    ctx.autotune(emb, W.nprobe)
    ld, se, per = ctx.logdet(emb, W.nprobe, W.nsteps, W.probe_seed, reorth=1)
    P = O.FFTProblem(W.n1, W.n2, problem["mask"], W.cov)
    _, _, ref = P.logdet(W.nprobe, W.nsteps, W.probe_seed, probe_ids=[0, W.nprobe - 1], reorth=True)
    assert per[0] == pytest.approx(ref[0], rel=1e-3)
    assert per[-1] == pytest.approx(ref[1], rel=1e-3)
    emb.free()


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


def test_loglik_krige_assembles_its_parts_at_full_size(problem):
    ctx = problem["ctx"]
    y, X = problem["y"], problem["X"]
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    opts = kry.Opts(prec=kry.KRY_F32, nprobe=W.nprobe, nsteps=W.nsteps, seed=W.probe_seed, rtol=W.cg_tol,
                    maxit=20000, reorth=1)
    cells = np.flatnonzero(~problem["mask"].ravel()).astype(np.int64)
    S1, S2 = I.cell_centres(W.n1, W.n2)
    Xc = I.covariates(S1.ravel()[cells], S2.ravel()[cells])
    res = ctx.loglik_krige(W.cov, opts, yt, Xt, cells=torch.tensor(cells, device=DEV),
                           Xc=torch.tensor(Xc.T.copy(), device=DEV))
    assert res["status"] == kry.KRY_OK
    # the same pieces through the separate entry points
    emb = ctx.embed(W.cov, kry.KRY_F32)
    ld, _, _ = ctx.logdet(emb, W.nprobe, W.nsteps, W.probe_seed, reorth=1)
    Z, _, _, st = ctx.solve(emb, torch.tensor(np.vstack([y, X.T]), device=DEV), rtol=W.cg_tol, maxit=20000)
    Z = Z.cpu().numpy()
    # GLS from the symmetrised Gram matrix of [y, X] and K^-1 [y, X] (symmetric in
    # exact arithmetic; the two triangles differ at the CG tolerance)
    A = X.T @ Z[1:].T
    g = 0.5 * (X.T @ Z[0] + Z[1:] @ y)
    beta = np.linalg.solve(0.5 * (A + A.T), g)
    quad = y @ Z[0] - beta @ g
    ll = -0.5 * (ld + quad + y.size * math.log(2 * math.pi))
    assert res["logdet"] == pytest.approx(ld, rel=1e-9)
    assert np.allclose(res["beta"], beta, rtol=1e-5, atol=1e-7)
    assert res["loglik"] == pytest.approx(ll, rel=1e-6)
    # the kriging means honour the trend at cells far from any data (here: all finite)
    mc = res["mean_cells"].cpu().numpy()
    assert np.all(np.isfinite(mc)) and mc.shape == (cells.size,)
    emb.free()


def test_bccb_logdet_at_full_size(problem):
    """BCCB log-det and range derivative of the grid1024 covariance (2048^2 torus) vs the oracle."""
    ld, dl = problem["ctx"].bccb_logdet(W.cov)
    ref_ld, ref_dl = O.bccb_logdet(W.n1, W.n2, W.cov, "scaled")
    assert ld == pytest.approx(ref_ld, rel=1e-9)
    assert dl == pytest.approx(ref_dl, rel=1e-7)
