"""FP64 CPU oracle for the Kryging hot path (Majumder, Guan, Reich & Saibaba, arXiv 2012.13133).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this module: only the test suite, the package smoke check and the benchmark's
CPU-baseline leg may use it.  It shares no code with the CUDA library; the two
meet only through the seeded inputs of ``paper_2012_13133_gb300.inputs``.

Everything here is plain, slow and FP64: dense covariance matrices and Cholesky
where sizes allow, explicit DFT matrices on tiny grids, and library FFTs
(scipy.fft) as a single step where sizes do not.  Each function names the
passage of the paper it follows.

Readings taken where the paper is silent (each one is listed in the design
notes of the repository):
  * grid cells are centred at ((i + 1/2)/n1, (j + 1/2)/n2) on the unit square;
  * the circulant embedding has size M_d = next power of two >= 2 n_d (the paper
    uses 2 n_d - 1), lags wrap to their minimal image and a lag of exactly M_d/2
    averages the two images;
  * the likelihood is the marginal Gaussian log-likelihood of the observed
    cells with beta profiled by GLS (the paper's exact profile likelihood,
    Eq. exact_plik, differs from it by 1/2 log det Gamma^{-1} plus a constant);
  * the log-determinant is the stochastic Lanczos quadrature estimate (the
    stochastic trace alternative of Sec. 3.3) with Rademacher probes drawn from
    splitmix64 counters;
  * the kriging variance is the simple-kriging variance (the quantity the
    bootstrap of Sec. 3.5, Eq. bootstrap_uq, estimates);
  * Alg. 1's beta_{i+1} step is read as ||A Sigma v_i - alpha_i u_i|| / tau, like
    beta_1, which U^T U = tau^2 I (Eq. exact_arith) requires;
  * the BCCB log-determinant of Sec. 3.3 is offered in two readings: "literal"
    (the (2n-1)-torus, first n1 x n2 frequencies) and "scaled" (the matvec's
    power-of-two torus, all frequencies, times n1 n2 / (M1 M2));
  * the Wendland weights of Sec. 2 are normalised over the cell centres that
    exist, so near the border of the grid a site may have fewer than four.

Parity of the paper's own tables is unpinned: they are replicate averages of
unpublished random data and fix no value of this path.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft
import scipy.linalg
import scipy.special

_WORKERS = max(1, int(os.environ.get("KRY_ORACLE_THREADS", os.cpu_count() or 1)))

# --------------------------------------------------------------------------------------
# Covariance model (Sec. 2, Matern correlation with sigma^2 outside; anisotropy per Sec. 2)
# --------------------------------------------------------------------------------------


def matern_bessel(r, nu):
    """Matern correlation from its Bessel-K definition (Sec. 2):
    2^(1-nu)/Gamma(nu) * (sqrt(2 nu) r)^nu * K_nu(sqrt(2 nu) r), r = d / range; 1 at r = 0."""
    r = np.asarray(r, dtype=np.float64)
    x = math.sqrt(2.0 * nu) * r
    out = np.ones_like(x)
    pos = x > 0
    xp = x[pos]
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        val = (2.0 ** (1.0 - nu) / scipy.special.gamma(nu)) * xp ** nu * scipy.special.kv(nu, xp)
    val = np.where(np.isfinite(val), val, 0.0)
    out[pos] = val
    return out


def matern(r, nu):
    """Matern correlation; closed forms for nu = 1/2, 3/2, 5/2 (the half-integer
    Bessel functions are elementary), the Bessel form otherwise."""
    r = np.asarray(r, dtype=np.float64)
    x = math.sqrt(2.0 * nu) * r
    if nu == 0.5:
        return np.exp(-x)
    if nu == 1.5:
        return (1.0 + x) * np.exp(-x)
    if nu == 2.5:
        return (1.0 + x + x * x / 3.0) * np.exp(-x)
    return matern_bessel(r, nu)


def scaled_distance(h1, h2, cov):
    """d / range for lag (h1, h2): rotate by the anisotropy angle, stretch the
    minor axis by the axis ratio (ratio 1 = Euclidean distance over range)."""
    h1 = np.asarray(h1, dtype=np.float64)
    h2 = np.asarray(h2, dtype=np.float64)
    ca, sa = math.cos(cov.angle), math.sin(cov.angle)
    u = ca * h1 + sa * h2
    v = -sa * h1 + ca * h2
    return np.sqrt(u * u + (cov.ratio * v) ** 2) / cov.range


def covariance(h1, h2, cov):
    """sigma^2 * rho(d) for lag (h1, h2), no nugget."""
    return cov.sigma2 * matern(scaled_distance(h1, h2, cov), cov.nu)


# --------------------------------------------------------------------------------------
# Dense forms (model Eq. obs_mod with A = row selection; covariance of Sec. 2)
# --------------------------------------------------------------------------------------


def coords(n1, n2):
    s1 = (np.arange(n1) + 0.5) / n1
    s2 = (np.arange(n2) + 0.5) / n2
    S1, S2 = np.meshgrid(s1, s2, indexing="ij")
    return S1, S2


def dense_sigma(sa, sb, cov):
    """sigma^2 Sigma between site sets sa (m,2) and sb (k,2), no nugget."""
    h1 = sa[:, None, 0] - sb[None, :, 0]
    h2 = sa[:, None, 1] - sb[None, :, 1]
    return covariance(h1, h2, cov)


def observed_sites(n1, n2, mask):
    S1, S2 = coords(n1, n2)
    return np.stack([S1[mask], S2[mask]], axis=1)


def dense_K(n1, n2, mask, cov):
    """Marginal covariance of the observed cells, K = sigma^2 A Sigma A^T + tau^2 I (Eq. obs_mod)."""
    s = observed_sites(n1, n2, mask)
    K = dense_sigma(s, s, cov)
    K[np.diag_indices_from(K)] += cov.tau2
    return K


# --------------------------------------------------------------------------------------
# Circulant embedding of the BTTB covariance (Sec. 3, Sec. 3.3, Appendix A Eq. circ_diag)
# --------------------------------------------------------------------------------------


def embed_size(n):
    """Smallest power of two >= 2 n."""
    M = 1
    while M < 2 * n:
        M *= 2
    return M


def lag_covariance(n1, n2, M1, M2, cov):
    """First row c of the block-circulant embedding on the M1 x M2 torus:
    c[j1, j2] = sigma^2 rho(l1/n1, l2/n2) with l the minimal image of j
    (j - M when j > M/2); at j = M/2 the two images +-M/2 are averaged."""
    def images(M):
        j = np.arange(M)
        a = np.where(2 * j <= M, j, j - M)        # image with j = M/2 -> +M/2
        b = np.where(2 * j < M, j, j - M)         # image with j = M/2 -> -M/2
        return a.astype(np.float64), b.astype(np.float64)
    a1, b1 = images(M1)
    a2, b2 = images(M2)
    dx1, dx2 = 1.0 / n1, 1.0 / n2
    c = np.zeros((M1, M2))
    for l1 in (a1, b1):
        for l2 in (a2, b2):
            c += covariance(l1[:, None] * dx1, l2[None, :] * dx2, cov)
    return 0.25 * c


def embedding_eigs(c):
    """Eigenvalues of the block-circulant embedding: the 2-D DFT of its first row (Eq. circ_diag)."""
    lam = scipy.fft.fft2(c, workers=_WORKERS)
    return lam.real, float(np.max(np.abs(lam.imag)))


def dft_matrix(M):
    j = np.arange(M)
    return np.exp(-2j * np.pi * np.outer(j, j) / M)


def bttb_matvec_dft(n1, n2, M1, M2, lam, mask, v, tau2):
    """K v by the circulant embedding with explicit DFT matrices (tiny grids only):
    scatter A^T v onto the M1 x M2 torus, DFT, multiply by the eigenvalues,
    inverse DFT, keep the grid, gather A, add the nugget."""
    F1, F2 = dft_matrix(M1), dft_matrix(M2)
    g = np.zeros((M1, M2))
    sub = np.zeros((n1, n2))
    sub[mask] = v
    g[:n1, :n2] = sub
    G = F1 @ g @ F2.T
    r = (np.conj(F1) @ (lam * G) @ np.conj(F2).T) / (M1 * M2)
    return r.real[:n1, :n2][mask] + tau2 * v


def sigma_conv_fft(n1, n2, M1, M2, lam, grid_vals):
    """(sigma^2 Sigma g) on the n1 x n2 grid for a grid vector g (batch in the leading axes), by FFT."""
    g = np.asarray(grid_vals)
    pad = np.zeros(g.shape[:-2] + (M1, M2))
    pad[..., :n1, :n2] = g
    out = scipy.fft.ifft2(lam * scipy.fft.fft2(pad, workers=_WORKERS), workers=_WORKERS)
    return out.real[..., :n1, :n2]


def bttb_matvec_fft(n1, n2, M1, M2, lam, mask, v, tau2):
    """K v for v of shape (p,) or (nvec, p), by FFT (library FFT as one step)."""
    v = np.asarray(v, dtype=np.float64)
    squeeze = v.ndim == 1
    V = v[None] if squeeze else v
    g = np.zeros((V.shape[0], n1, n2))
    g[:, mask] = V
    out = sigma_conv_fft(n1, n2, M1, M2, lam, g)[:, mask] + tau2 * V
    return out[0] if squeeze else out


# --------------------------------------------------------------------------------------
# Rademacher probes from splitmix64 counters (Steele, Lea & Flood 2014)
# --------------------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """splitmix64 output function applied to state x (state advanced by the golden gamma first)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def rademacher_probe(seed, k, p):
    """z_k[i] = +1 if bit 63 of splitmix64(seed XOR (k * 2^32 + i)) is 0, else -1."""
    i = np.arange(p, dtype=np.uint64)
    key = np.uint64(seed) ^ ((np.uint64(k) << np.uint64(32)) | i)
    bit = splitmix64(key) >> np.uint64(63)
    return np.where(bit == 0, 1.0, -1.0)


# --------------------------------------------------------------------------------------
# Stochastic Lanczos quadrature for log det K (Sec. 3.3, stochastic trace alternative)
# --------------------------------------------------------------------------------------


def lanczos(matvec, z, m, reorth=False):
    """m steps of symmetric Lanczos from q1 = z/||z||.  Stops early when
    beta_j < 1e-12 |alpha_1|.  Returns alpha (length k) and beta (length k-1).

    reorth=False is the recurrence as the paper runs it for its results (the
    basis is not reorthogonalised, Sec. 3.2).  reorth=True orthogonalises each
    new vector against every earlier one (classical Gram-Schmidt, applied
    twice), the reorthogonalisation Sec. 3.2 leaves to the user: the
    tridiagonal is then, up to rounding, the exact-arithmetic one, i.e. the
    Jacobi matrix of the m-point Gauss rule of the spectral measure of z."""
    q = z / np.linalg.norm(z)
    q_prev = np.zeros_like(q)
    b_prev = 0.0
    basis = [q]
    alpha, beta = [], []
    for j in range(m):
        u = matvec(q)
        a = float(q @ u)
        w = u - a * q - b_prev * q_prev
        alpha.append(a)
        if reorth:
            Q = np.array(basis)
            for _ in range(2):
                w = w - Q.T @ (Q @ w)
        b = float(np.linalg.norm(w))
        if j == m - 1:
            break
        if b < 1e-12 * abs(alpha[0]):
            break
        beta.append(b)
        q_prev, q, b_prev = q, w / b, b
        if reorth:
            basis.append(q)
    return np.array(alpha), np.array(beta)


def gauss_quadrature_logdet(alpha, beta, znorm2):
    """||z||^2 sum_j tau_j^2 log theta_j over the eigenpairs (theta_j, first
    eigenvector components tau_j) of the Lanczos tridiagonal (Golub-Welsch)."""
    if len(alpha) == 1:
        return znorm2 * math.log(alpha[0])
    theta, U = scipy.linalg.eigh_tridiagonal(alpha, beta)
    return znorm2 * float(np.sum(U[0] ** 2 * np.log(theta)))


def slq_logdet(matvec, p, nprobe, nsteps, seed, probes=None, reorth=False):
    """SLQ estimate of log det K: mean over probes of the Gauss quadrature of
    z^T log(K) z.  ``probes`` overrides the Rademacher probes (e.g. the unit
    vectors, for which the sum over all p probes is exact up to quadrature error);
    ``reorth`` as in ``lanczos``.  Returns (estimate, standard error, per-probe values)."""
    vals = []
    for k in range(nprobe):
        z = rademacher_probe(seed, k, p) if probes is None else probes(k)
        a, b = lanczos(matvec, z, nsteps, reorth)
        vals.append(gauss_quadrature_logdet(a, b, float(z @ z)))
    vals = np.array(vals)
    se = float(np.std(vals, ddof=1) / math.sqrt(nprobe)) if nprobe > 1 else 0.0
    return float(np.mean(vals)), se, vals


# --------------------------------------------------------------------------------------
# Conjugate gradients (replaces the O(n^3) solves, Sec. 3)
# --------------------------------------------------------------------------------------


def cg(matvec, b, tol=1e-10, maxit=100000):
    """Plain CG from x0 = 0 until ||r|| <= tol ||b||.  Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0:
        return x, 0
    for it in range(1, maxit + 1):
        Ap = matvec(p)
        a = rr / float(p @ Ap)
        x += a * p
        r -= a * Ap
        rr_new = float(r @ r)
        if math.sqrt(rr_new) <= tol * bnorm:
            return x, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxit


def pcg(matvec, precond, b, tol=1e-10, maxit=100000):
    """Preconditioned CG from x0 = 0 with the stopping rule of ``cg`` (||r|| <= tol ||b||):
    z = M^-1 r, alpha = r^T z / p^T A p, x += alpha p, r -= alpha A p, p = z + (r'^T z' / r^T z) p.
    For symmetric positive definite A and M^-1 it converges to the same solution A^-1 b as plain
    CG (the solves of Sec. 3 need only matvecs).  Returns (x, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0:
        return x, 0
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    for it in range(1, maxit + 1):
        Ap = matvec(p)
        a = rz / float(p @ Ap)
        x += a * p
        r -= a * Ap
        if math.sqrt(float(r @ r)) <= tol * bnorm:
            return x, it
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


# --------------------------------------------------------------------------------------
# Profile log-likelihood and kriging
# --------------------------------------------------------------------------------------


def gls_loglik(logdet, Kinv_y, Kinv_X, y, X):
    """GLS beta and the marginal log-likelihood with beta profiled:
    beta = (X^T K^-1 X)^-1 X^T K^-1 y, r = y - X beta,
    l = -1/2 [log det K + r^T K^-1 r + p log 2 pi]."""
    A = X.T @ Kinv_X
    g = X.T @ Kinv_y
    beta = np.linalg.solve(A, g)
    quad = float(y @ Kinv_y - beta @ g)
    p = y.shape[0]
    ll = -0.5 * (logdet + quad + p * math.log(2.0 * math.pi))
    return ll, beta, quad


def loglik_dense(K, y, X):
    """Marginal log-likelihood by Cholesky (exact log det)."""
    L = scipy.linalg.cho_factor(K, lower=True)
    logdet = 2.0 * float(np.sum(np.log(np.diag(L[0]))))
    Kinv_y = scipy.linalg.cho_solve(L, y)
    Kinv_X = scipy.linalg.cho_solve(L, X)
    ll, beta, quad = gls_loglik(logdet, Kinv_y, Kinv_X, y, X)
    return dict(loglik=ll, beta=beta, logdet=logdet, quad=quad)


def krige_dense(n1, n2, mask, cov, y, X, targets, X_t, beta=None):
    """Universal-kriging mean at target sites (m,2) with covariates X_t, and the
    simple-kriging variance sigma^2 - c_t^T K^-1 c_t (c_t = sigma^2 Sigma_{o,t}):
    mu_t = X_t beta + c_t^T K^-1 (y - X beta)  (the paper's x-hat, Eq. act_xhat, plus the trend)."""
    s = observed_sites(n1, n2, mask)
    K = dense_K(n1, n2, mask, cov)
    L = scipy.linalg.cho_factor(K, lower=True)
    if beta is None:
        beta = loglik_dense(K, y, X)["beta"]
    w = scipy.linalg.cho_solve(L, y - X @ beta)
    C = dense_sigma(np.asarray(targets), s, cov)          # (m, p)
    mean = X_t @ beta + C @ w
    var = cov.sigma2 - np.einsum("ij,ji->i", C, scipy.linalg.cho_solve(L, C.T))
    return mean, var


class FFTProblem:
    """A masked grid problem with the FP64 circulant-embedding matvec (Sec. 3)."""

    def __init__(self, n1, n2, mask, cov):
        self.n1, self.n2, self.mask, self.cov = n1, n2, np.asarray(mask, bool), cov
        self.M1, self.M2 = embed_size(n1), embed_size(n2)
        c = lag_covariance(n1, n2, self.M1, self.M2, cov)
        self.lam, self.imag = embedding_eigs(c)
        self.c0 = c[0, 0]
        self.p = int(self.mask.sum())

    def matvec(self, v):
        return bttb_matvec_fft(self.n1, self.n2, self.M1, self.M2, self.lam, self.mask, v, self.cov.tau2)

    def sigma_at(self, v, cells):
        """(sigma^2 Sigma A^T v) at linear cell indices ``cells`` (no nugget)."""
        g = np.zeros((self.n1, self.n2))
        g[self.mask] = v
        return sigma_conv_fft(self.n1, self.n2, self.M1, self.M2, self.lam, g).ravel()[cells]

    def torus_inverse(self, v):
        """A (S + tau^2 I)^-1 A^T v with S the circulant embedding of sigma^2 Sigma on the M1 x M2
        torus: the inverse of the torus covariance plus nugget, restricted to the observed cells
        (eigenvalues 1 / (max(Lambda, 0) + tau^2) in the FFT basis; a CG preconditioner)."""
        lam_inv = 1.0 / (np.maximum(self.lam, 0.0) + self.cov.tau2)
        g = np.zeros((self.n1, self.n2))
        g[self.mask] = v
        return sigma_conv_fft(self.n1, self.n2, self.M1, self.M2, lam_inv, g)[self.mask]

    def solve(self, B, tol=1e-10, precond=False):
        """K^-1 B by CG (precond=True: CG preconditioned by ``torus_inverse``, same solution)."""
        B = np.asarray(B, dtype=np.float64)

        def one(b):
            return pcg(self.matvec, self.torus_inverse, b, tol) if precond else cg(self.matvec, b, tol)

        if B.ndim == 1:
            return one(B)
        cols, its = zip(*(one(B[:, j]) for j in range(B.shape[1])))
        return np.stack(cols, axis=1), max(its)

    def logdet(self, nprobe, nsteps, seed, probe_ids=None, reorth=False):
        ids = range(nprobe) if probe_ids is None else probe_ids
        vals = []
        for k in ids:
            z = rademacher_probe(seed, k, self.p)
            a, b = lanczos(self.matvec, z, nsteps, reorth)
            vals.append(gauss_quadrature_logdet(a, b, float(z @ z)))
        vals = np.array(vals)
        se = float(np.std(vals, ddof=1) / math.sqrt(len(vals))) if len(vals) > 1 else 0.0
        return float(np.mean(vals)), se, vals

    def profile_loglik(self, y, X, nprobe, nsteps, seed, tol=1e-10, reorth=False):
        ld, se, _ = self.logdet(nprobe, nsteps, seed, reorth=reorth)
        sol, _ = self.solve(np.column_stack([y, X]), tol)
        ll, beta, quad = gls_loglik(ld, sol[:, 0], sol[:, 1:], y, X)
        return dict(loglik=ll, beta=beta, logdet=ld, logdet_se=se, quad=quad)

    def krige_cells(self, y, X, beta, cells, X_t, tol=1e-10):
        w, _ = cg(self.matvec, y - X @ beta, tol)
        return X_t @ beta + self.sigma_at(w, cells)


# --------------------------------------------------------------------------------------
# BCCB log-determinant approximation (Sec. 3.3) and its range derivative (Appendix A,
# Eq. circ_diag and Eq. trace_approx)
# --------------------------------------------------------------------------------------


def matern_dr(r, nu):
    """d/dr of the Matern correlation rho_nu(r) (Sec. 2).  Closed forms for nu = 1/2, 3/2,
    5/2 (x = sqrt(2 nu) r: -e^-x; -sqrt(3) x e^-x; -sqrt(5) x (1 + x) e^-x / 3); otherwise
    d/dx [x^nu K_nu(x)] = -x^nu K_{nu-1}(x) (DLMF 10.29.4) gives
    -2^(1-nu)/Gamma(nu) sqrt(2 nu) x^nu K_{nu-1}(x)."""
    r = np.asarray(r, dtype=np.float64)
    s = math.sqrt(2.0 * nu)
    x = s * r
    if nu == 0.5:
        return -np.exp(-x)
    if nu == 1.5:
        return -s * x * np.exp(-x)
    if nu == 2.5:
        return -s * x * (1.0 + x) * np.exp(-x) / 3.0
    out = np.zeros_like(x)
    pos = x > 0
    xp = x[pos]
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        val = -(2.0 ** (1.0 - nu) / scipy.special.gamma(nu)) * s * xp ** nu * scipy.special.kv(nu - 1.0, xp)
    out[pos] = np.where(np.isfinite(val), val, 0.0)
    if nu < 0.5:
        out[~pos] = -np.inf
    elif nu == 0.5:
        out[~pos] = -1.0
    return out


def covariance_drange(h1, h2, cov):
    """d/d(range) of sigma^2 rho(d / range): with r = d / range, dr / d(range) = -r / range."""
    r = scaled_distance(h1, h2, cov)
    return cov.sigma2 * matern_dr(r, cov.nu) * (-r / cov.range)


def _torus_first_row(n1, n2, M1, M2, cov, fn):
    """First row of the block-circulant extension on an M1 x M2 torus of the BTTB matrix with
    entries fn(lag): minimal-image lags, the two images of a lag of exactly M/2 averaged
    (no such lag on an odd torus)."""
    def images(M):
        j = np.arange(M)
        a = np.where(2 * j <= M, j, j - M)
        b = np.where(2 * j < M, j, j - M)
        return a.astype(np.float64), b.astype(np.float64)
    a1, b1 = images(M1)
    a2, b2 = images(M2)
    c = np.zeros((M1, M2))
    for l1 in (a1, b1):
        for l2 in (a2, b2):
            c += fn(l1[:, None] / n1, l2[None, :] / n2, cov)
    return 0.25 * c


def bccb_logdet(n1, n2, cov, reading="scaled", floor_rel=2.220446049250313e-16):
    """Approximate log det Sigma(theta) of the n1 x n2 BTTB covariance (no nugget) and its
    derivative dL with respect to the range, from the eigenvalues D1 of a block-circulant
    extension and D2 of the extension of d Sigma / d(range) (Eq. circ_diag): log det ~ sum
    log D1, dL ~ sum D2 / D1 (Eq. trace_approx).  Readings of Sec. 3.3's formula:

      "literal": the paper's (2 n1 - 1) x (2 n2 - 1) extension, frequencies p < n1, q < n2
                 (the formula's sums over p = 1..n1, q = 1..n2 with omega = exp(-2 pi i/(2n-1)));
      "scaled":  the matvec's power-of-two M1 x M2 extension, all frequencies, scaled by
                 n1 n2 / (M1 M2).

    Eigenvalues below floor_rel * max are reset to that value before the log (the
    "forcefully resetting" recourse of Sec. 3.6) and contribute no derivative term.
    Returns (logdet, dL)."""
    N = n1 * n2
    if reading == "literal":
        M1, M2 = 2 * n1 - 1, 2 * n2 - 1
    elif reading == "scaled":
        M1, M2 = embed_size(n1), embed_size(n2)
    else:
        raise ValueError(reading)
    d1 = scipy.fft.fft2(_torus_first_row(n1, n2, M1, M2, cov, covariance), workers=_WORKERS).real
    d2 = scipy.fft.fft2(_torus_first_row(n1, n2, M1, M2, cov, covariance_drange), workers=_WORKERS).real
    if reading == "literal":
        d1, d2, scale = d1[:n1, :n2], d2[:n1, :n2], 1.0
    else:
        scale = N / float(M1 * M2)
    f = floor_rel * float(d1.max())
    keep = d1 > f
    ld = scale * float(np.sum(np.log(np.where(keep, d1, f))))
    dl = scale * float(np.sum(np.where(keep, d2 / np.where(keep, d1, 1.0), 0.0)))
    return ld, dl


# --------------------------------------------------------------------------------------
# Circulant-embedding sampling (bootstrap of Sec. 3.5; negative-eigenvalue caveat of Sec. 3.6)
# --------------------------------------------------------------------------------------


def sample_embed_size(n1, n2, cov, max_doublings=3):
    """Smallest power-of-two torus (>= 2n per axis, doubled up to ``max_doublings``
    times) whose embedding eigenvalues satisfy min >= -1e-10 max."""
    M1, M2 = embed_size(n1), embed_size(n2)
    for _ in range(max_doublings + 1):
        lam, _ = embedding_eigs(lag_covariance(n1, n2, M1, M2, cov))
        if lam.min() >= -1e-10 * lam.max():
            return M1, M2
        M1, M2 = 2 * M1, 2 * M2
    return M1 // 2, M2 // 2


def sample_field(n1, n2, M1, M2, cov, xi):
    """One Gaussian-process sample on the n1 x n2 grid: the real part of
    FFT2( sqrt(max(Lambda, 0) / (M1 M2)) * (xi[0] + i xi[1]) ), cropped.  Small
    negative eigenvalues are reset to zero (Sec. 3.6 caveat)."""
    lam, _ = embedding_eigs(lag_covariance(n1, n2, M1, M2, cov))
    lam = np.maximum(lam, 0.0)
    z = np.sqrt(lam / (M1 * M2)) * (xi[0] + 1j * xi[1])
    return scipy.fft.fft2(z, workers=_WORKERS).real[:n1, :n2]


def gengk(n1, n2, mask, cov, b, k, reorth=False):
    """Generalized Golub-Kahan bidiagonalization (Alg. 1) for the genHyBR problem of Sec. 3.2:
    A = selection of the observed cells of the n1 x n2 grid, Sigma = the correlation matrix
    (sigma^2 = 1) applied on the whole grid by the FP64 circulant-embedding matvec, b = y - X beta,
    R = tau^2 I.  Reading of a garble in the algorithm's step for beta_{i+1}: beta_{i+1} =
    ||A Sigma v_i - alpha_i u_i||_2 / tau (as beta_1 = ||b||_2 / tau), which is what makes
    U^T U = tau^2 I hold (Eq. exact_arith).  reorth: re-orthogonalise each new u against U
    (Euclidean) and each new v against V (Sigma inner product), twice.
    Returns (beta1, U[p, k+1], V[N, k+1], alphas[k+1], betas[k+1] with betas[0] = beta1)."""
    mask = np.asarray(mask, bool)
    full = np.ones((n1, n2), bool)
    corr = type(cov)(1.0, cov.range, cov.nu, 0.0, cov.angle, cov.ratio)
    M1, M2 = embed_size(n1), embed_size(n2)
    lam, _ = embedding_eigs(lag_covariance(n1, n2, M1, M2, corr))

    def sig(v):                                   # Sigma v on the whole grid
        return bttb_matvec_fft(n1, n2, M1, M2, lam, full, v, 0.0)

    def At(u):                                    # A^T u: observed values into a zero grid
        g = np.zeros(n1 * n2)
        g[mask.ravel()] = u
        return g

    tau2 = cov.tau2
    tau = math.sqrt(tau2)
    N, p = n1 * n2, int(mask.sum())
    U = np.zeros((p, k + 1))
    V = np.zeros((N, k + 1))
    SV = np.zeros((N, k + 1))
    alphas, betas = np.zeros(k + 1), np.zeros(k + 1)
    beta1 = float(np.linalg.norm(b)) / tau
    U[:, 0] = b / beta1
    betas[0] = beta1
    w = At(U[:, 0]) / tau2
    sw = sig(w)
    alphas[0] = math.sqrt(float(w @ sw))
    V[:, 0], SV[:, 0] = w / alphas[0], sw / alphas[0]
    for i in range(k):
        t = SV[mask.ravel(), i] - alphas[i] * U[:, i]
        if reorth:
            for _ in range(2):
                t -= U[:, : i + 1] @ (U[:, : i + 1].T @ t) / tau2
        betas[i + 1] = float(np.linalg.norm(t)) / tau
        U[:, i + 1] = t / betas[i + 1]
        w = At(U[:, i + 1]) / tau2 - betas[i + 1] * V[:, i]
        if reorth:
            for _ in range(2):
                w -= V[:, : i + 1] @ (SV[:, : i + 1].T @ w)
        sw = sig(w)
        alphas[i + 1] = math.sqrt(float(w @ sw))
        V[:, i + 1], SV[:, i + 1] = w / alphas[i + 1], sw / alphas[i + 1]
    return beta1, U, V, alphas, betas


def genhybr(n1, n2, mask, cov, b, k, reorth=False):
    """genHyBR estimate of x_hat (Sec. 3.2): with B_k the (k+1) x k lower bidiagonal of alphas
    and betas from Alg. 1, z_k = (B_k^T B_k + I / sigma^2)^-1 B_k^T beta1 e_1 and
    x_k* = Sigma V_k z_k (Eq. xhat_est), Sigma the correlation; x_hat^T Sigma^-1 x_hat ~ ||z_k||^2.
    Returns dict(x, z, psi2 = ||b - A x_k*||^2, z2 = ||z_k||^2)."""
    mask = np.asarray(mask, bool)
    beta1, U, V, al, be = gengk(n1, n2, mask, cov, b, k, reorth)
    Bk = np.zeros((k + 1, k))
    for i in range(k):
        Bk[i, i] = al[i]
        Bk[i + 1, i] = be[i + 1]
    rhs = Bk.T @ (beta1 * np.eye(k + 1)[:, 0])
    z = np.linalg.solve(Bk.T @ Bk + np.eye(k) / cov.sigma2, rhs)
    corr = type(cov)(1.0, cov.range, cov.nu, 0.0, cov.angle, cov.ratio)
    M1, M2 = embed_size(n1), embed_size(n2)
    lam, _ = embedding_eigs(lag_covariance(n1, n2, M1, M2, corr))
    q = V[:, :k] @ z
    x = bttb_matvec_fft(n1, n2, M1, M2, lam, np.ones((n1, n2), bool), q, 0.0)
    psi = b - x[mask.ravel()]
    return dict(x=x, z=z, q=q, psi=psi, psi2=float(psi @ psi), z2=float(z @ z))


def approx_profile_loglik(n1, n2, mask, cov, b, k, reading="scaled", reorth=False):
    """The paper's approximate profile log-likelihood (Eq. prof_lik), constants dropped as there:
    -p/2 log tau^2 - ||psi_k*||^2 / (2 tau^2) - n/2 log sigma^2 - 1/2 logdet~ Sigma - ||z_k||^2 / (2 sigma^2),
    Sigma the correlation, logdet~ its BCCB approximation (Sec. 3.3, reading as bccb_logdet)."""
    mask = np.asarray(mask, bool)
    g = genhybr(n1, n2, mask, cov, b, k, reorth)
    corr = type(cov)(1.0, cov.range, cov.nu, 0.0, cov.angle, cov.ratio)
    ld, _ = bccb_logdet(n1, n2, corr, reading)
    p, N = int(mask.sum()), n1 * n2
    pl = (-0.5 * p * math.log(cov.tau2) - g["psi2"] / (2 * cov.tau2) - 0.5 * N * math.log(cov.sigma2) - 0.5 * ld -
          g["z2"] / (2 * cov.sigma2))
    return dict(pl=pl, logdet=ld, **g)


def approx_gradient(n1, n2, mask, cov, b, k, reading="scaled", reorth=False):
    """The paper's approximate gradient of the profile log-likelihood (Appendix A, Eq. approx_grad),
    in its parametrisation lambda^2 = 1/sigma^2, lambda_e^2 = 1/tau^2:
      d pl / d lambda^2   ~ n / (2 lambda^2) - ||z_k||^2 / 2,
      d pl / d rho        ~ -dL~ / 2 + lambda^2 / 2 (V_k z_k)^T dSigma (V_k z_k),
      d pl / d lambda_e^2 ~ p / (2 lambda_e^2) - ||psi_k*||^2 / 2,
    (d pl / d beta ~ lambda_e^2 X^T psi_k*, formed by the caller from the returned psi), with
    dSigma the range derivative of the correlation applied by its circulant extension on the whole
    grid and dL~ the BCCB derivative of Sec. 3.3 (reading as bccb_logdet).
    Returns dict(grad = [d/d lambda^2, d/d rho, d/d lambda_e^2], psi)."""
    mask = np.asarray(mask, bool)
    g = genhybr(n1, n2, mask, cov, b, k, reorth)
    corr = type(cov)(1.0, cov.range, cov.nu, 0.0, cov.angle, cov.ratio)
    M1, M2 = embed_size(n1), embed_size(n2)
    lam_d = scipy.fft.fft2(_torus_first_row(n1, n2, M1, M2, corr, covariance_drange), workers=_WORKERS).real
    dq = bttb_matvec_fft(n1, n2, M1, M2, lam_d, np.ones((n1, n2), bool), g["q"], 0.0)
    _, dl = bccb_logdet(n1, n2, corr, reading)
    lam2, lame2 = 1.0 / cov.sigma2, 1.0 / cov.tau2
    N, p = n1 * n2, int(mask.sum())
    grad = [N / (2 * lam2) - 0.5 * g["z2"], -0.5 * dl + 0.5 * lam2 * float(g["q"] @ dq),
            p / (2 * lame2) - 0.5 * g["psi2"]]
    return dict(grad=np.array(grad), psi=g["psi"])


def bootstrap_kriging_variance(n1, n2, mask, cov, targets, xis, epss):
    """Parametric-bootstrap MSE of the kriging prediction of x at grid cells ``targets`` (flat
    row-major indices), theta and beta known (Sec. 3.5, Eq. bootstrap_uq): replicate b draws
    x_b from the white noise xis[b] with the circulant-embedding sampler, forms
    y_b - X beta = A x_b + tau eps_b (epss[b]: p standard normals), predicts
    x_hat_b = sigma^2 Sigma_{t,o} K^-1 (y_b - X beta) and the estimate is
    mean_b (x_b(t) - x_hat_b(t))^2.  The MSE of y at a target adds tau^2 (its nugget noise is
    independent of everything else)."""
    mask = np.asarray(mask, bool)
    M1, M2 = xis.shape[-2:]
    K = dense_K(n1, n2, mask, cov)
    L = scipy.linalg.cho_factor(K, lower=True)
    S1, S2 = coords(n1, n2)
    t_sites = np.stack([S1.ravel()[targets], S2.ravel()[targets]], axis=1)
    C = dense_sigma(t_sites, observed_sites(n1, n2, mask), cov)        # (m, p)
    acc = np.zeros(len(targets))
    for xi, eps in zip(xis, epss):
        x = sample_field(n1, n2, M1, M2, cov, xi)
        w = scipy.linalg.cho_solve(L, x[mask] + math.sqrt(cov.tau2) * eps)
        acc += (x.ravel()[targets] - C @ w) ** 2
    return acc / len(xis)


def make_data(n1, n2, mask, cov, beta, xi, eps):
    """y = X beta + x(obs) + tau eps with x the circulant-embedding GP sample of
    white noise ``xi`` (shape (2, M1, M2); Eq. obs_mod with A = row selection).
    The noise is drawn by the caller from the shared seeded generators."""
    M1, M2 = xi.shape[1], xi.shape[2]
    x = sample_field(n1, n2, M1, M2, cov, xi)
    S1, S2 = coords(n1, n2)
    X = np.stack([np.ones(int(mask.sum())), S1[mask], S2[mask]], axis=1)
    y = X @ np.asarray(beta, dtype=np.float64) + x[mask] + math.sqrt(cov.tau2) * eps
    return y, X, x


# --------------------------------------------------------------------------------------
# Irregular observation sites: the Wendland mapping matrix A of Sec. 2
# --------------------------------------------------------------------------------------


def wendland(d):
    """Wendland's compactly supported function w(d) = (1 - d)_+^4 (1 + 4 d) (Sec. 2)."""
    d = np.asarray(d, dtype=np.float64)
    return np.where(d < 1.0, (1.0 - d) ** 4 * (1.0 + 4.0 * d), 0.0)


def wendland_A_dense(n1, n2, sites):
    """The p x n mapping matrix of Sec. 2, written out over every grid cell: the distance of site
    i to cell centre j is d_ij = max(|s_i1 - s*_j1| / Delta_1, |s_i2 - s*_j2| / Delta_2) in grid
    spacings (Delta_d = 1 / n_d), and A_ij = w(d_ij) / sum_k w(d_ik).  Cells are numbered row-major
    (j = j1 n2 + j2).  O(p n): for small grids."""
    sites = np.asarray(sites, dtype=np.float64)
    S1, S2 = coords(n1, n2)
    d = np.maximum(np.abs(sites[:, None, 0] - S1.ravel()[None, :]) * n1,
                   np.abs(sites[:, None, 1] - S2.ravel()[None, :]) * n2)
    w = wendland(d)
    return w / w.sum(axis=1, keepdims=True)


def wendland_A(n1, n2, sites):
    """The same matrix in sparse triplet form: only the cell centres within one spacing of a site
    on both axes (at most 2 x 2 of them) have d_ij < 1, so only they are visited.  Returns
    (rows, cols, vals) with rows sorted, as int64, int64, float64 arrays."""
    sites = np.asarray(sites, dtype=np.float64)
    rows, cols, vals = [], [], []
    for i, (a, b) in enumerate(sites):
        u1, u2 = a * n1 - 0.5, b * n2 - 0.5          # site in cell-centre index units
        cand = [(j1, j2) for j1 in (math.floor(u1), math.floor(u1) + 1)
                for j2 in (math.floor(u2), math.floor(u2) + 1)
                if 0 <= j1 < n1 and 0 <= j2 < n2]
        ws = [float(wendland(max(abs(u1 - j1), abs(u2 - j2)))) for j1, j2 in cand]
        tot = sum(ws)
        for (j1, j2), wv in zip(cand, ws):
            if wv > 0.0:
                rows.append(i)
                cols.append(j1 * n2 + j2)
                vals.append(wv / tot)
    return np.array(rows, np.int64), np.array(cols, np.int64), np.array(vals)


def wendland_dense_K(n1, n2, sites, cov):
    """Marginal covariance of irregular sites, K = sigma^2 A Sigma A^T + tau^2 I (Eq. obs_mod with
    the Wendland A), from the dense covariance of the whole latent grid."""
    A = wendland_A_dense(n1, n2, sites)
    S1, S2 = coords(n1, n2)
    g = np.stack([S1.ravel(), S2.ravel()], axis=1)
    K = A @ dense_sigma(g, g, cov) @ A.T
    K[np.diag_indices_from(K)] += cov.tau2
    return K


class IrregularProblem:
    """Irregular sites on an n1 x n2 latent grid (Sec. 2): K v = sigma^2 A Sigma A^T v + tau^2 v
    with A in sparse form and Sigma applied by the FP64 circulant-embedding FFT on the whole grid
    (Sec. 3)."""

    def __init__(self, n1, n2, sites, cov):
        self.n1, self.n2, self.cov = n1, n2, cov
        self.sites = np.asarray(sites, dtype=np.float64)
        self.p = self.sites.shape[0]
        self.rows, self.cols, self.vals = wendland_A(n1, n2, self.sites)
        self.M1, self.M2 = embed_size(n1), embed_size(n2)
        self.lam, _ = embedding_eigs(lag_covariance(n1, n2, self.M1, self.M2, cov))

    def A(self, x):
        """A x for a whole-grid vector x (row-major)."""
        out = np.zeros(self.p)
        np.add.at(out, self.rows, self.vals * x[self.cols])
        return out

    def At(self, v):
        """A^T v as a whole-grid vector."""
        out = np.zeros(self.n1 * self.n2)
        np.add.at(out, self.cols, self.vals * v[self.rows])
        return out

    def sigma(self, x):
        """sigma^2 Sigma x on the whole grid."""
        return sigma_conv_fft(self.n1, self.n2, self.M1, self.M2, self.lam,
                              x.reshape(self.n1, self.n2)).ravel()

    def matvec(self, v):
        return self.A(self.sigma(self.At(v))) + self.cov.tau2 * v

    def profile_loglik(self, y, X, nprobe, nsteps, seed, tol=1e-10, reorth=False):
        vals = []
        for k in range(nprobe):
            z = rademacher_probe(seed, k, self.p)
            a, b = lanczos(self.matvec, z, nsteps, reorth)
            vals.append(gauss_quadrature_logdet(a, b, float(z @ z)))
        ld = float(np.mean(vals))
        cols = [cg(self.matvec, c, tol)[0] for c in np.column_stack([y, X]).T]
        ll, beta, quad = gls_loglik(ld, cols[0], np.stack(cols[1:], axis=1), y, X)
        return dict(loglik=ll, beta=beta, logdet=ld, quad=quad)

    def krige_grid(self, y, X, beta, X_grid, tol=1e-10):
        """Mean of y at every latent cell (A = identity row there): X_grid beta + x_hat, with
        x_hat = sigma^2 Sigma A^T K^-1 (y - X beta) (Eq. act_xhat by the Woodbury identity)."""
        w, _ = cg(self.matvec, y - X @ beta, tol)
        return X_grid @ beta + self.sigma(self.At(w))
