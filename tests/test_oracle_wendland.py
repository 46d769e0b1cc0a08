"""Pins of the oracle's irregular-site path (Sec. 2: the Wendland mapping matrix A), CPU only."""
import math

import numpy as np
import pytest
import scipy.integrate

from oracle import kryoracle as O
from paper_2012_13133_gb300 import inputs as I

COV = I.Cov(1.0, 0.2, 1.5, 0.1)


def test_wendland_function_values_shape_and_integral():
    assert O.wendland(0.0) == 1.0
    assert O.wendland(1.0) == 0.0 and O.wendland(1.7) == 0.0
    assert O.wendland(0.5) == pytest.approx(0.5 ** 4 * 3.0, rel=1e-15)
    # C^2 at the support's edge and flat at the origin: w'(d) = -20 d (1 - d)^3
    h = 1e-6
    for d in (0.0 + h, 0.3, 0.7, 1.0 - h):
        fd = (O.wendland(d + h) - O.wendland(d - h)) / (2 * h)
        assert fd == pytest.approx(-20 * d * (1 - d) ** 3, abs=1e-8)
    # integral over the support: int_0^1 t^4 (5 - 4 t) dt = 1 - 2/3
    val, _ = scipy.integrate.quad(lambda d: float(O.wendland(d)), 0.0, 1.0)
    assert val == pytest.approx(1.0 / 3.0, rel=1e-12)
    d = np.linspace(0.0, 1.0, 101)
    assert np.all(np.diff(O.wendland(d)) <= 0)


def test_mapping_rows_on_and_between_grid_points():
    n1, n2 = 8, 10
    S1, S2 = O.coords(n1, n2)
    # a site on a cell centre: the mapping is exact (a unit row)
    A = O.wendland_A_dense(n1, n2, [[S1[3, 4], S2[3, 4]]])
    assert A[0, 3 * n2 + 4] == 1.0 and np.count_nonzero(A) == 1
    # the centre of four cell centres: four equal weights
    s = [[(S1[3, 4] + S1[4, 4]) / 2, (S2[3, 4] + S2[3, 5]) / 2]]
    A = O.wendland_A_dense(n1, n2, s)
    nz = np.flatnonzero(A[0])
    assert sorted(nz) == sorted([3 * n2 + 4, 4 * n2 + 4, 3 * n2 + 5, 4 * n2 + 5])
    assert np.allclose(A[0, nz], 0.25, rtol=0, atol=1e-15)
    # halfway between two centres of one row: two equal weights (the others lie at distance 1)
    s = [[S1[2, 6], (S2[2, 6] + S2[2, 7]) / 2]]
    A = O.wendland_A_dense(n1, n2, s)
    nz = np.flatnonzero(A[0])
    assert sorted(nz) == [2 * n2 + 6, 2 * n2 + 7] and np.allclose(A[0, nz], 0.5, atol=1e-15)


def test_sparse_mapping_equals_the_written_out_definition():
    n1, n2 = 12, 9
    rng = np.random.default_rng(4)
    sites = np.vstack([rng.random((200, 2)),
                       [[0.0, 0.0], [1.0, 1.0], [0.01, 0.99], [0.5, 0.0]]])   # corners and edges
    A = O.wendland_A_dense(n1, n2, sites)
    r, c, v = O.wendland_A(n1, n2, sites)
    B = np.zeros_like(A)
    B[r, c] = v
    assert np.abs(A - B).max() <= 1e-14          # the two forms round the distances differently
    assert np.all(A >= 0) and np.allclose(A.sum(axis=1), 1.0, atol=1e-15)
    assert (A > 0).sum(axis=1).max() <= 4


def test_sites_at_cell_centres_reduce_to_the_gridded_model():
    n1, n2 = 10, 12
    mask = I.mask_uniform(n1, n2, 0.3, 8)
    sites = O.observed_sites(n1, n2, mask)
    K_irr = O.wendland_dense_K(n1, n2, sites, COV)
    K_grid = O.dense_K(n1, n2, mask, COV)
    assert np.abs(K_irr - K_grid).max() <= 1e-14


def irregular_case(n1=16, n2=14, p=150, seed=9):
    rng = np.random.default_rng(seed)
    sites = rng.random((p, 2))
    X = np.column_stack([np.ones(p), sites])
    y = X @ np.array([1.0, 0.5, -0.5]) + rng.standard_normal(p)
    return n1, n2, sites, X, y


def test_fft_matvec_equals_dense_marginal_covariance():
    n1, n2, sites, _, _ = irregular_case()
    P = O.IrregularProblem(n1, n2, sites, COV)
    K = O.wendland_dense_K(n1, n2, sites, COV)
    V = np.random.default_rng(10).standard_normal((sites.shape[0], 3))
    for j in range(3):
        out = P.matvec(V[:, j])
        assert np.linalg.norm(out - K @ V[:, j]) <= 1e-12 * np.linalg.norm(K @ V[:, j])


def test_irregular_gls_and_kriging_equal_dense_cholesky():
    n1, n2, sites, X, y = irregular_case()
    P = O.IrregularProblem(n1, n2, sites, COV)
    K = O.wendland_dense_K(n1, n2, sites, COV)
    ref = O.loglik_dense(K, y, X)
    res = P.profile_loglik(y, X, nprobe=4, nsteps=30, seed=1)
    assert np.allclose(res["beta"], ref["beta"], rtol=1e-8, atol=1e-10)
    assert res["quad"] == pytest.approx(ref["quad"], rel=1e-8)
    # kriging means at every latent cell: X_g beta + sigma^2 Sigma_{g,g} A^T K^-1 (y - X beta)
    S1, S2 = O.coords(n1, n2)
    g = np.stack([S1.ravel(), S2.ravel()], axis=1)
    Xg = np.column_stack([np.ones(n1 * n2), g])
    A = O.wendland_A_dense(n1, n2, sites)
    beta = ref["beta"]
    dense = Xg @ beta + O.dense_sigma(g, g, COV) @ A.T @ np.linalg.solve(K, y - X @ beta)
    got = P.krige_grid(y, X, beta, Xg)
    assert np.abs(got - dense).max() <= 1e-8 * np.abs(dense).max()


def test_slq_on_the_irregular_operator_matches_cholesky_with_unit_probes():
    """Gauss quadrature with the unit vectors e_i as probes sums to log det K exactly (the
    quadrature is exact once the Krylov space is full)."""
    n1, n2, sites, _, _ = irregular_case(n1=8, n2=8, p=40)
    P = O.IrregularProblem(n1, n2, sites, COV)
    K = O.wendland_dense_K(n1, n2, sites, COV)
    tot = 0.0
    for i in range(P.p):
        e = np.zeros(P.p)
        e[i] = 1.0
        a, b = O.lanczos(P.matvec, e, P.p, reorth=True)
        tot += O.gauss_quadrature_logdet(a, b, 1.0)
    assert tot == pytest.approx(np.linalg.slogdet(K)[1], rel=1e-9)
    assert math.isfinite(tot)
