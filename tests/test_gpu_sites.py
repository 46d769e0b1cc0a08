"""Irregular observation sites (Sec. 2, the Wendland mapping matrix A) through the C ABI,
against the FP64 oracle's IrregularProblem.

Workload shape of the paper's third simulation: 40,000 sites uniform on the unit square
over latent grids of 200 x 200 and 400 x 400 cells, exponential covariance with
sigma^2 = 3, tau^2 = 0.5, range 0.1 (the paper's simulation parameters), trend
X = [1, s1, s2].  The data are the oracle's: the latent field is its circulant-embedding
sample of seeded white noise, y = X beta + A x + tau eps.

Checked: K v (FP64 1e-12, FP32 1e-5 relative l2), the profile log-likelihood and
log det with the same probes (1e-3 relative; the oracle's Lanczos basis is fully
reorthogonalised, the library's partially), beta, and the kriging means at every
latent cell (1e-4 relative l2); the entry points that need a mask refuse sites."""
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
COV = I.Cov(3.0, 0.1, 0.5, 0.5)
BETA = (1.0, 0.5, -0.5)
NSITE = 40000


def _sites(seed=31):
    return I.uniform_sites(NSITE, seed)


def _oracle_data(n1, n2, sites, P):
    M1, M2 = O.sample_embed_size(n1, n2, COV)
    xi, eps = I.data_noise(M1, M2, sites.shape[0], 41)
    x = O.sample_field(n1, n2, M1, M2, COV, xi)
    X = I.covariates(sites[:, 0], sites[:, 1])
    y = X @ np.array(BETA) + P.A(x.ravel()) + math.sqrt(COV.tau2) * eps
    return X, y


@pytest.mark.parametrize("n", [200, 400])
@pytest.mark.parametrize("prec", [kry.KRY_F64, kry.KRY_F32])
def test_sites_matvec_matches_oracle(n, prec):
    sites = _sites()
    P = O.IrregularProblem(n, n, sites, COV)
    ctx = kry.Context(0)
    assert ctx.set_sites(torch.tensor(sites, device=DEV), n, n) == NSITE
    emb = ctx.embed(COV, prec)
    V = I.normals((5, NSITE), 32)
    dt = torch.float64 if prec == kry.KRY_F64 else torch.float32
    out = ctx.matvec(emb, torch.tensor(V, dtype=dt, device=DEV)).double().cpu().numpy()
    ref = np.stack([P.matvec(v) for v in V])
    tol = 1e-12 if prec == kry.KRY_F64 else 1e-5
    for k in range(V.shape[0]):
        err = np.linalg.norm(out[k] - ref[k]) / np.linalg.norm(ref[k])
        assert err <= tol, (n, prec, k, err)
    emb.free()
    ctx.close()


def test_sites_matvec_border_and_clustered_sites():
    """Sites on the domain's edges and corners (fewer than four cell centres), and many sites
    sharing cells: FP64 matvec against the oracle."""
    n = 64
    rng = np.random.default_rng(5)
    edge = np.array([[0.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 0.0], [0.5, 0.0], [0.0, 0.37], [1.0, 0.81],
                     [0.5 / n, 0.5 / n], [1 - 0.5 / n, 0.3]])
    cluster = 0.4 + 0.01 * rng.random((300, 2))
    sites = np.vstack([edge, cluster, rng.random((700, 2))])
    P = O.IrregularProblem(n, n, sites, COV)
    ctx = kry.Context(0)
    ctx.set_sites(torch.tensor(sites, device=DEV), n, n)
    emb = ctx.embed(COV, kry.KRY_F64)
    V = I.normals((3, sites.shape[0]), 33)
    out = ctx.matvec(emb, torch.tensor(V, device=DEV)).cpu().numpy()
    for k in range(3):
        ref = P.matvec(V[k])
        assert np.linalg.norm(out[k] - ref) / np.linalg.norm(ref) <= 1e-12
    emb.free()
    ctx.close()


@pytest.mark.parametrize("prec", [kry.KRY_F64, kry.KRY_F32])
def test_sites_loglik_and_grid_kriging_match_oracle(prec):
    n = 200
    sites = _sites()
    P = O.IrregularProblem(n, n, sites, COV)
    X, y = _oracle_data(n, n, sites, P)
    nprobe, nsteps = 16, 40
    ref = P.profile_loglik(y, X, nprobe, nsteps, 7, tol=1e-10, reorth=True)
    S1, S2 = I.cell_centres(n, n)
    Xg = I.covariates(S1.ravel(), S2.ravel())
    ref_mean = P.krige_grid(y, X, ref["beta"], Xg, tol=1e-10)

    ctx = kry.Context(0)
    ctx.set_sites(torch.tensor(sites, device=DEV), n, n)
    yt, Xt = torch.tensor(y, device=DEV), torch.tensor(X.T.copy(), device=DEV)
    opts = kry.Opts(prec=prec, nprobe=nprobe, nsteps=nsteps, seed=7, rtol=1e-10 if prec == kry.KRY_F64 else 1e-7,
                    maxit=20000, reorth=1)
    cells = torch.arange(n * n, dtype=torch.int64, device=DEV)
    res = ctx.loglik_krige(COV, opts, yt, Xt, cells=cells, Xc=torch.tensor(Xg.T.copy(), device=DEV))
    assert res["status"] == kry.KRY_OK
    e_ll = abs(res["loglik"] - ref["loglik"]) / abs(ref["loglik"])
    e_ld = abs(res["logdet"] - ref["logdet"]) / abs(ref["logdet"])
    e_b = np.linalg.norm(res["beta"] - ref["beta"]) / np.linalg.norm(ref["beta"])
    mc = res["mean_cells"].cpu().numpy()
    e_m = np.linalg.norm(mc - ref_mean) / np.linalg.norm(ref_mean)
    print(f"sites {n}^2, prec {prec}: loglik {e_ll:.2e}, logdet {e_ld:.2e}, beta {e_b:.2e}, means {e_m:.2e}")
    assert e_ll <= 1e-3 and e_ld <= 1e-3
    assert e_b <= 1e-4
    assert e_m <= 1e-4
    # the batched-setting path (two settings in shared launches) gives the same log-likelihood
    other = I.Cov(3.0, 0.05, 0.5, 0.5)
    both = ctx.profile_loglik(yt, Xt, [COV, other], opts)
    assert both["loglik"][0] == pytest.approx(res["loglik"], rel=1e-6)
    ctx.close()


def test_sites_refuse_mask_only_entry_points():
    n = 32
    sites = I.uniform_sites(500, 3)
    ctx = kry.Context(0)
    ctx.set_sites(torch.tensor(sites, device=DEV), n, n)
    y = torch.tensor(I.normals(500, 1), device=DEV)
    X = torch.tensor(I.covariates(sites[:, 0], sites[:, 1]).T.copy(), device=DEV)
    cells = torch.arange(10, dtype=torch.int64, device=DEV)
    Xc = torch.ones((3, 10), dtype=torch.float64, device=DEV)
    with pytest.raises(kry.KryError) as ei:
        ctx.krige(COV, kry.Opts(prec=kry.KRY_F64), y, X, cells=cells, Xc=Xc, variances=True)
    assert ei.value.status == kry.KRY_EUNSUPPORTED
    bad = torch.tensor([[0.5, 0.5], [1.5, 0.2]], dtype=torch.float64, device=DEV)
    with pytest.raises(kry.KryError) as ei:
        ctx.set_sites(bad, n, n)
    assert ei.value.status == kry.KRY_EINVAL
    ctx.close()
