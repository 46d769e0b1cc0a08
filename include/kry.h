/*
 * kry.h -- C ABI of the Kryging hot path on one GB300 (sm_103a).
 *
 * Kryging (Majumder, Guan, Reich & Saibaba, arXiv 2012.13133) models gridded
 * spatial data as y = X beta + A x + eps (Sec. 2, Eq. obs_mod) with a latent
 * Gaussian process x ~ N(0, sigma^2 Sigma) under a Matern correlation (Sec. 2)
 * and nugget eps ~ N(0, tau^2 I).  A is a row selection: the observation mask.
 * The library computes, with hand-written CUDA kernels and no CPU fallback:
 *
 *   - the eigenvalues of the block-circulant embedding of the BTTB covariance
 *     (Sec. 3 and Sec. 3.3; Appendix A, Eq. circ_diag);
 *   - the marginal covariance matvec K v = sigma^2 A Sigma A^T v + tau^2 v by
 *     scatter, 2-D FFT, eigenvalue multiply, inverse FFT, gather (Sec. 3);
 *   - log det K by stochastic Lanczos quadrature (the stochastic trace
 *     alternative named in Sec. 3.3);
 *   - CG solves with K (the matvec-only solves of Sec. 3), the GLS profile
 *     log-likelihood and kriging means and variances (Sec. 3.1, Eq. act_xhat;
 *     Sec. 3.5);
 *   - Gaussian-process samples by circulant embedding (Sec. 3.5 bootstrap;
 *     the negative-eigenvalue caveat of Sec. 3.6).
 *
 * Conventions shared by every entry point:
 *   Status     Every function returns kry_status; nothing throws across the
 *              ABI.  On failure kry_last_error(ctx) holds a one-line message.
 *              Arguments are validated before any launch.
 *   Memory     The caller owns every data buffer it passes; "_dev" pointers are
 *              device pointers on the context's device, others host pointers.
 *              The library owns kry_ctx, kry_embed and their scratch, released
 *              by kry_destroy / kry_embed_free.
 *   Streams    All work is enqueued on the context's stream.  Calls that
 *              return scalars through host pointers synchronise that stream;
 *              kry_matvec does not.
 *   Threads    A context is not thread-safe; use one context per host thread.
 *   Layout     The grid is n1 x n2, row-major (row index i along the first
 *              coordinate), cell (i, j) centred at ((i + 1/2) dx1, (j + 1/2) dx2).
 *              Observed cells are numbered 0..p-1 in row-major order; a
 *              "vector" is p values in that order.  Batches of vectors are
 *              column-major with leading dimension ld >= p.
 *   Precision  KRY_F32: FP32 vectors and FFTs, FP64 Krylov scalars (alpha,
 *              beta, dot products, quadrature).  KRY_F64: FP64 throughout.
 *              Solves always take and return FP64 vectors; with KRY_F32 they
 *              run FP32 CG whose solution accumulates in FP64 and whose
 *              residual is periodically replaced by the true FP64 residual.
 */
#ifndef KRY_H
#define KRY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KRY_OK = 0,
    KRY_EINVAL = 1,       /* bad argument (sizes, parameters, null pointers) */
    KRY_ENOMEM = 2,       /* device allocation failed */
    KRY_ENOTPSD = 3,      /* embedding not positive semi-definite where that is required */
    KRY_ENOCONV = 4,      /* CG reached maxit before rtol; partial results written */
    KRY_ENAN = 5,         /* a reduction produced NaN/Inf */
    KRY_ETIMEOUT = 6,     /* a bounded device wait gave up */
    KRY_ECUDA = 7,        /* a CUDA runtime call failed */
    KRY_EUNSUPPORTED = 8  /* valid request outside the supported sizes */
} kry_status;

/* KRY_AUTO (kry_opts only; embeddings take KRY_F32 or KRY_F64): FP32 for each
 * covariance setting FP32 resolves, FP64 for the others (see kry_opts). */
typedef enum { KRY_F32 = 0, KRY_F64 = 1, KRY_AUTO = 2 } kry_prec;

/* Regular grid on the unit square (Sec. 4 layout): n1 x n2 cells of size dx1 x dx2. */
typedef struct {
    int32_t n1, n2;
    double dx1, dx2;
} kry_grid;

/* Covariance sigma2 * Matern_nu(d / range) + tau2 * I (Sec. 2).  d is the
 * Euclidean lag after rotating by aniso_angle (radians, counter-clockwise
 * from the first axis) and stretching the minor axis by aniso_ratio
 * (geometric anisotropy, Sec. 2; aniso_ratio = 1 is isotropic). */
typedef struct {
    double sigma2, range, nu, tau2;
    double aniso_angle, aniso_ratio;
} kry_cov;

/* Krylov settings.  nprobe Rademacher probes x nsteps Lanczos steps for the
 * log-determinant; CG to true relative residual rtol (maxit iterations at most
 * per right-hand side).  reorth: 0 = the Lanczos basis is not
 * reorthogonalised (as the paper runs it for its results, Sec. 3.2); 1 =
 * partial reorthogonalisation (Sec. 3.2 leaves a scheme to the user; see
 * kry_logdet), which keeps every basis vector on the device
 * (nprobe * nsteps * p values: FP16 for FP32 embeddings, FP64 otherwise).  precond: 0 =
 * plain CG; 1 = CG preconditioned by M^-1 = A (S + tau2 I)^-1 A^T, S the
 * circulant embedding of sigma2 Sigma on the matvec's torus (its inverse is
 * diagonal in the same FFT basis, so M^-1 costs one more FFT matvec per
 * iteration).  It pays where most of the grid is observed and the gaps are
 * clustered (cloud-like masks), not under scattered missing cells; it applies
 * to FP32 solves of one covariance setting with tau2 > 0 on an observation
 * mask, and is ignored otherwise (with irregular sites, close sites make
 * A (S + tau2 I)^-1 A^T nearly singular).  2 = automatic: preconditioned when
 * at least 0.4 of the observed cells have all four grid neighbours observed
 * (kry_mask_interior; on 512^2 masks that is where the preconditioned solve
 * was the faster one).  The result does not depend on it beyond the CG
 * tolerance.
 * prec: KRY_F32 runs FP32 vectors and matvecs with FP64 scalars (CG
 * convergence is still judged on the FP64 true residual, and a solve that
 * stalls returns KRY_ENOCONV); KRY_F64 runs FP64 throughout.  KRY_AUTO, in
 * kry_profile_loglik, kry_krige, kry_loglik_krige and kry_bootstrap_var,
 * runs FP32 for each covariance setting whose conditioning FP32 resolves,
 * kappa = (max |Lambda| + tau2) / tau2 <= 4e6 (every eigenvalue of K lies in
 * [tau2, max |Lambda| + tau2]; FP32 CG stalls as kappa u32 nears one, u32 =
 * 2^-24), and FP64 for a setting above that bound or with tau2 = 0, alone
 * (kry_promoted counts them).  FP64 costs far more on large ill-conditioned
 * grids: a 2000-request serving stream that took 615 s on one slot in FP32
 * took 2418 s with KRY_AUTO.  In FP32 the log-determinant wants reorth = 1:
 * without it the FP32 quadrature drifts as kappa grows (measured 8.6e-4
 * relative at kappa 3.3e5 on a 1024^2 grid, 5.6e-3 on 256^2 with the same
 * range in cells), while with it, or in FP64 either way, it stays within
 * 1e-5 of the reorthogonalised FP64 value. */
typedef struct {
    kry_prec prec;
    int32_t nprobe, nsteps;
    uint64_t seed;
    double rtol;
    int32_t maxit;
    int32_t reorth;
    int32_t precond;
} kry_opts;

typedef struct kry_ctx kry_ctx;       /* opaque, library-owned */
typedef struct kry_embed kry_embed;   /* opaque, library-owned */

/* Create a context on CUDA device `device` using `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  *ctx is NULL on failure. */
kry_status kry_create(kry_ctx** ctx, int device, void* cuda_stream);
void kry_destroy(kry_ctx* ctx);
/* Last error message of ctx ("" if none); valid until the next call on ctx. */
const char* kry_last_error(const kry_ctx* ctx);

/* Observation pattern A (Sec. 2: a subset of identity rows).  mask_dev holds
 * n1*n2 bytes, row-major, nonzero = observed.  Builds the library's index
 * lists on the device and returns the number of observed cells p in *p_out.
 * Requires 4 <= n1, n2 <= 4096 and p >= 1.  Synchronises the stream. */
kry_status kry_set_mask(kry_ctx* ctx, const kry_grid* grid, const uint8_t* mask_dev, int64_t* p_out);

/* Share of the observed cells of the last kry_set_mask whose four grid
 * neighbours are observed too (a neighbour beyond the grid edge counts as
 * observed): near 1 for clustered gaps, about (1 - missing share)^4 for
 * scattered holes; 0 without a mask or with sites.  It decides
 * kry_opts.precond = 2.  (No counterpart in the paper.) */
kry_status kry_mask_interior(kry_ctx* ctx, double* interior);

/* Number of covariance settings that calls on ctx with prec = KRY_AUTO ran in
 * FP64 because FP32 would not resolve their conditioning (kry_opts, prec),
 * counted since kry_create. */
kry_status kry_promoted(kry_ctx* ctx, int64_t* count);

/* Irregular observation sites (Sec. 2: y = X beta + A x + eps with A the
 * p x n mapping matrix of Wendland weights).  sites_dev holds nsite (x1, x2)
 * FP64 pairs, row-major, inside the domain [0, n1 dx1] x [0, n2 dx2]; the
 * latent field x lives on the cell centres of grid.  Row i of A weights the
 * cell centres c_j within one spacing of site s_i along both axes (at most
 * 2 x 2 of them) by w(d_ij) / sum_k w(d_ik), w(d) = (1 - d)^4 (1 + 4 d) for
 * d < 1, d_ij = max(|s_i1 - c_j1| / dx1, |s_i2 - c_j2| / dx2); near the border
 * the centres that exist are normalised over.  A is built on the device by
 * site and by cell (its transpose, each cell's entries in site order, so
 * results do not depend on scheduling).  Afterwards p = nsite and every
 * matvec, log-determinant, solve, likelihood and kriging call on ctx uses
 * K = sigma2 A Sigma A^T + tau2 I (Sigma applied on the whole grid by the
 * FFT passes); kriging covers grid cells (the mean of y at a cell: trend plus
 * the latent prediction there), without variances or off-grid targets;
 * kry_bootstrap_var, kry_genhybr and kry_matvec_noalloc need a mask and return
 * KRY_EUNSUPPORTED.  kry_set_mask replaces the sites.  Errors: KRY_EINVAL for
 * a site outside the domain or bad arguments, KRY_EUNSUPPORTED for grid sides
 * outside [4, 4096].  Synchronises the stream. */
kry_status kry_set_sites(kry_ctx* ctx, const kry_grid* grid, const double* sites_dev, int64_t nsite);

/* Eigenvalues of the block-circulant embedding of sigma2 * Sigma on the
 * M1 x M2 torus, M_d = smallest power of two >= 2 n_d (Sec. 3.3; Eq. circ_diag).
 * The lag covariance is evaluated in FP64 (closed forms for nu in {1/2, 3/2,
 * 5/2}, Bessel K_nu otherwise), transformed by a 2-D FFT in FP64 and kept on
 * the device in FP64 (and FP32 when prec = KRY_F32).  No eigenvalue is
 * clamped: the matvec is exact whatever their sign (Sec. 3.6 caveat).
 * *min_over_max receives min(Lambda) / max(Lambda) (may be NULL).  Uses the
 * grid of the last kry_set_mask.  Synchronises the stream. */
kry_status kry_embed_eigs(kry_ctx* ctx, const kry_cov* cov, kry_prec prec,
                          kry_embed** out, double* min_over_max);
void kry_embed_free(kry_embed* e);

/* out = K v for nvec vectors (K = sigma2 A Sigma A^T + tau2 I, Sec. 3).  v_dev
 * and out_dev are FP32 (prec KRY_F32) or FP64 (KRY_F64) arrays of nvec columns
 * with leading dimension ld.  Asynchronous.  v_dev and out_dev must not overlap. */
kry_status kry_matvec(kry_ctx* ctx, const kry_embed* e, const void* v_dev, void* out_dev,
                      int32_t nvec, int64_t ld);

/* Allocation-free form of kry_matvec (the paper has no counterpart; this is a
 * deployment aid).  Same arguments and result as kry_matvec, for callers that
 * cannot allocate device memory at call time: applications whose device
 * memory is all owned by their own pool or arena (cudaMalloc would fail or
 * fragment it), and latency-critical loops that cannot absorb the
 * device-wide synchronisation of cudaMalloc / cudaFree.  It runs the same FFT
 * passes under the same launch schedule as kry_matvec, so on the same context
 * the two agree bit for bit; only the FFT intermediate differs: it lives in a
 * 16 MiB static device array of the library (held by every GPU that loads it,
 * until exit) and is filled as many complex pairs at a time as fit.  Hence
 * n1 * M2 * sizeof(complex) must not exceed 16 MiB (grids up to 1024 x 1024
 * in FP32, 1024 x 512 in FP64); larger grids return KRY_EUNSUPPORTED with a
 * message.  The call performs no allocation itself; ctx, its mask and e must
 * be set up beforehand (their creation allocates).  The first call on a
 * device (and the first after that device's CUDA context changes, e.g. after
 * cudaDeviceReset) looks up the array's device address: make it before any
 * stream capture.  All calls on a device share the array and it keeps the
 * last call's contents: calls that overlap on the GPU race, so the caller
 * must serialise them.  Asynchronous. */
kry_status kry_matvec_noalloc(kry_ctx* ctx, const kry_embed* e, const void* v_dev, void* out_dev,
                              int32_t nvec, int64_t ld);

/* Stochastic Lanczos quadrature estimate of log det K (Sec. 3.3, stochastic
 * trace alternative): probe k has entries z_k[i] = +1 if bit 63 of
 * splitmix64(seed XOR (k * 2^32 + i)) is 0, else -1; nsteps Lanczos steps
 * from q1 = z/||z||, stopping early when beta_j < 1e-12 |alpha_1|; Gauss
 * quadrature ||z||^2 sum_j tau_j^2 log theta_j of the tridiagonal.
 * reorth = 0: plain three-term recurrence (the paper's runs, Sec. 3.2).
 * reorth = 1: partial reorthogonalisation (Simon 1984): per probe, estimates
 * of the basis' loss of orthogonality are carried by a scalar recurrence whose
 * rounding term is that of the FFT matvec (unit roundoff x log2(M1 M2)) and,
 * when one exceeds sqrt(unit roundoff) of the embedding's precision, the new
 * basis vector and the next are orthogonalised against all earlier ones (a
 * second Gram-Schmidt pass when the first cancels most of the vector; for
 * FP32 embeddings the passes read an FP16 copy of the normalised basis, whose
 * rounding leaves components of about 2 unit roundoffs); the result then
 * follows the exact-arithmetic Gauss rule, which the plain FP32 recurrence
 * misses by ~1e-3 on ill-conditioned K.  The quadrature nodes are taken as
 * max(theta_j, tau2): every eigenvalue of K, and so every Ritz value of exact
 * arithmetic, is at least tau2.  *logdet = mean over
 * probes, *stderr_out = standard error (NULL allowed), per_probe[nprobe] the
 * per-probe values (host, NULL allowed).  Synchronises the stream. */
kry_status kry_logdet(kry_ctx* ctx, const kry_embed* e, int32_t nprobe, int32_t nsteps,
                      uint64_t seed, int32_t reorth, double* logdet, double* stderr_out,
                      double* per_probe);

/* Solve K X = B for nrhs FP64 right-hand sides (column-major, leading
 * dimension ld) by CG from X = 0 until the true residual satisfies
 * ||B - K X|| <= rtol ||B|| per column.  FP64 embeddings run FP64 CG.  FP32
 * embeddings run FP32 CG (FP32 matvec, FP64 scalars) with the solution
 * accumulated in FP64 and the recursive residual replaced by the true
 * residual from the FP64 matvec whenever it has fallen 10x or reached rtol
 * (reliable updates; convergence is judged on true residuals only).
 * iters (host, may be NULL) receives the largest per-column iteration count,
 * relres (host, may be NULL) the largest final true relative residual.
 * Returns KRY_ENOCONV, with X filled, when rtol was not reached within maxit
 * iterations.  Synchronises the stream. */
kry_status kry_solve(kry_ctx* ctx, const kry_embed* e, const double* B_dev, double* X_dev,
                     int32_t nrhs, int64_t ld, double rtol, int32_t maxit,
                     int32_t* iters, double* relres);

/* kry_solve preconditioned by M^-1 = A (S + tau2 I)^-1 A^T (S the circulant
 * embedding of sigma2 Sigma on the matvec's torus, whose inverse the same FFT
 * passes apply; see kry_opts.precond).  Same arguments, convergence test and
 * errors as kry_solve; the result agrees with it to the CG tolerance.  Each
 * iteration costs two FFT matvecs, so it pays where the iteration count falls
 * by more than half: masks with clustered gaps.  FP64 embeddings, tau2 = 0 and
 * irregular sites (kry_set_sites) run plain CG.  Library scratch: one more FP32 vector per right-hand side and
 * the preconditioner's eigenvalues (16 M1 M2 bytes) for the call. */
kry_status kry_solve_pre(kry_ctx* ctx, const kry_embed* e, const double* B_dev, double* X_dev, int32_t nrhs,
                         int64_t ld, double rtol, int32_t maxit, int32_t* iters, double* relres);

/* Marginal log-likelihood of the observed cells with beta profiled by GLS,
 * for ntheta covariance settings:
 *   beta = (X^T K^-1 X)^-1 X^T K^-1 y,  r = y - X beta,
 *   loglik = -1/2 [log det K + r^T K^-1 r + p log 2 pi],
 * log det K by kry_logdet's estimator (opts->nprobe, nsteps, seed), the solves
 * by kry_solve (opts->rtol, maxit).  It equals the paper's exact
 * profile likelihood (Eq. exact_plik) minus 1/2 log det Gamma^-1 and a
 * constant.  y_dev: p FP64; X_dev: p x ncov FP64 column-major (1 <= ncov <= 8).
 * Host outputs: loglik[ntheta], beta[ntheta * ncov], logdet[ntheta],
 * logdet_se[ntheta] (the last three may be NULL).  Synchronises the stream. */
kry_status kry_profile_loglik(kry_ctx* ctx, const double* y_dev, const double* X_dev, int32_t ncov,
                              const kry_cov* thetas, int32_t ntheta, const kry_opts* opts,
                              double* loglik, double* beta, double* logdet, double* logdet_se);

/* Kriging at target cells and at off-grid sites with beta from GLS:
 *   mean_t = X_t beta + sigma2 Sigma_{t,obs} K^-1 (y - X beta)
 * (the paper's x-hat of Eq. act_xhat plus the trend), and optionally the
 * simple-kriging variance sigma2 - sigma2^2 c_t^T K^-1 c_t at the target cells
 * (the quantity the bootstrap of Sec. 3.5 estimates).
 * cells_dev: ncell int64 row-major cell indices; Xc_dev: ncell x ncov FP64
 * column-major; sites_dev: nsite x 2 FP64 row-major coordinates; Xs_dev: nsite x
 * ncov.  Outputs (device, FP64): mean_cells_dev[ncell], mean_sites_dev[nsite],
 * var_cells_dev[ncell] (NULL skips the variances; their solves K^-1 c_t run 32
 * targets at a time, preconditioned as the [y, X] solve when opts->precond
 * applies).  beta_out (host, ncov, may be NULL).  Synchronises the stream. */
kry_status kry_krige(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts,
                     const double* y_dev, const double* X_dev, int32_t ncov,
                     const int64_t* cells_dev, const double* Xc_dev, int64_t ncell,
                     const double* sites_dev, const double* Xs_dev, int64_t nsite,
                     double* mean_cells_dev, double* mean_sites_dev, double* var_cells_dev,
                     double* beta_out);

/* One evaluation for one covariance setting: the profile log-likelihood of
 * kry_profile_loglik (log det K by SLQ, GLS beta, loglik) together with the
 * kriging means (and optional variances) of kry_krige, sharing one embedding
 * and one solve of K^-1 [y, X] (the kriging weights K^-1 (y - X beta) follow
 * from it without another solve).  Arguments as in those two calls; loglik,
 * beta[ncov], logdet and logdet_se are host outputs (all but loglik may be
 * NULL).  Synchronises the stream. */
kry_status kry_loglik_krige(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts,
                            const double* y_dev, const double* X_dev, int32_t ncov,
                            const int64_t* cells_dev, const double* Xc_dev, int64_t ncell,
                            const double* sites_dev, const double* Xs_dev, int64_t nsite,
                            double* mean_cells_dev, double* mean_sites_dev, double* var_cells_dev,
                            double* loglik, double* beta, double* logdet, double* logdet_se);

/* Circulant-embedding sample of the latent process on the n1 x n2 grid of the
 * last kry_set_mask (Sec. 3.5 bootstrap): out = Re FFT2( sqrt(max(Lambda, 0) /
 * (M1 M2)) * (xi_re + i xi_im) ) cropped to the grid, with the embedding on an
 * M1 x M2 torus (powers of two, each >= 2 n_d and <= 8192).  xi_dev holds 2 *
 * M1 * M2 FP64 normals (real plane, then imaginary plane); out_dev n1 * n2 FP64.
 * Negative eigenvalues are reset to zero (Sec. 3.6 caveat).  Asynchronous. */
kry_status kry_sample(kry_ctx* ctx, const kry_cov* cov, int32_t M1, int32_t M2,
                      const double* xi_dev, double* out_dev);

/* genHyBR estimate of the latent field and the paper's approximate profile
 * log-likelihood (Sec. 3.2, Alg. 1, Eq. xhat_est, Eq. prof_lik), for the
 * mask's grid, cov's sigma2, range, nu, anisotropy and nugget tau2 (> 0), and
 * b_dev = y - X beta on the p observed cells (device, FP64; the caller chooses
 * beta).  k steps of the generalized Golub-Kahan bidiagonalization (Alg. 1)
 * with A the observed-cell selection, Sigma the correlation matrix applied on
 * the whole grid by the FP64 embedding matvec and R = tau2 I, then
 * z_k = (B_k^T B_k + I / sigma2)^-1 B_k^T beta1 e1, x_k* = Sigma V_k z_k and
 *   *pl = -p/2 log tau2 - ||b - A x_k*||^2 / (2 tau2) - n/2 log sigma2
 *         - 1/2 logdet~ Sigma - ||z_k||^2 / (2 sigma2)
 * (constants dropped as in the paper; n = n1 n2; logdet~ the BCCB
 * approximation of kry_bccb_logdet).  beta_{i+1} of Alg. 1 is read as
 * ||A Sigma v_i - alpha_i u_i||_2 / tau (as beta_1 = ||b||_2 / tau), which
 * U^T U = tau2 I requires; no reorthogonalisation (as the paper runs it).
 * A step whose beta or alpha falls below 1e-13 of beta1 or alpha1 ends the
 * bidiagonalization early (the Krylov space then holds the solution; the
 * remaining alphas / betas are 0).
 * Outputs (each may be NULL): x_dev[n1 n2] (device) = x_k*; alphas[k+1],
 * betas[k+1] (host) the bidiagonal entries (betas[0] = beta1); *z2 =
 * ||z_k||^2, *psi2 = ||b - A x_k*||^2, *pl; grad[3] (host) the approximate
 * gradient of Appendix A (Eq. approx_grad) in the paper's parametrisation
 * lambda^2 = 1/sigma2, lambda_e^2 = 1/tau2:
 *   grad[0] = d pl / d lambda^2   ~ n / (2 lambda^2) - ||z_k||^2 / 2,
 *   grad[1] = d pl / d range      ~ -dL~ / 2 + lambda^2 / 2 (V_k z_k)^T dSigma (V_k z_k),
 *   grad[2] = d pl / d lambda_e^2 ~ p / (2 lambda_e^2) - ||psi_k*||^2 / 2
 * (dSigma the range derivative of the correlation, dL~ the BCCB derivative
 * of kry_bccb_logdet); psi_dev[p] (device) = psi_k* = b - A x_k*, from which
 * the caller forms d pl / d beta ~ lambda_e^2 X^T psi_k*.  Library scratch:
 * (2k + 6) n1 n2 doubles.  Errors: KRY_EINVAL (bad arguments, tau2 or sigma2
 * not positive, b zero), KRY_ENAN for a non-finite alpha or beta.
 * Synchronises the stream. */
kry_status kry_genhybr(kry_ctx* ctx, const kry_cov* cov, const double* b_dev, int32_t k, double* x_dev,
                       double* alphas, double* betas, double* z2, double* psi2, double* pl, double* grad,
                       double* psi_dev);

/* kry_genhybr in a chosen arithmetic.  prec = KRY_F64 is kry_genhybr itself.
 * prec = KRY_F32 keeps the Krylov vectors u_i, v_i and Sigma v_i in FP32 and
 * applies Sigma by the FP32 whole-grid embedding matvec, while every norm and
 * inner product of Alg. 1 (alpha_i, beta_i, w^T Sigma w), the projected
 * problem, ||z_k||^2, ||psi_k*||^2, pl and the gradient are accumulated and
 * kept in FP64; x_dev and psi_dev are written in FP64 from the FP32 vectors.
 * Without reorthogonalisation the recurrence amplifies rounding once
 * orthogonality is lost, and FP32 rounding is 2^29 times larger: measured
 * against the FP64 oracle, pl agrees to 4e-5 (40 x 36 grid, k = 15), 4e-7
 * (128^2, k = 30) and 8e-4 (1024^2, k = 50), and with the FP64 path to
 * 1.1e-4 at 4096^2 (k = 50), where it runs 6.6 times faster (0.18 s vs
 * 1.17 s).  reorth = 1 (beyond the paper) reorthogonalises each new u
 * against u_1..u_i (Euclidean, U^T U = tau2 I) and each new w against
 * v_1..v_i (Sigma inner product, through the stored Sigma v_j), by two
 * classical Gram-Schmidt passes, which keeps the recurrence on the exact
 * bidiagonal at O(k^2 n) extra work and (k + 1) n1 n2 more scratch:
 * measured against the oracle's reorthogonalised Alg. 1 (128^2, k = 40), the
 * bidiagonal to 1e-14 (FP64) and 4e-6 (FP32), pl to 4e-13 and 6e-8; at
 * 1024^2 (k = 50) FP32 took 92 ms and FP64 128 ms, pl equal to 6e-10.
 * Library scratch: (2k + 6) n1 n2 floats (FP32) or doubles (FP64), (3k + 7)
 * with reorth.  Arguments, outputs and errors as for kry_genhybr, plus
 * KRY_EINVAL for another prec or reorth.  Synchronises the stream. */
kry_status kry_genhybr_prec(kry_ctx* ctx, const kry_cov* cov, kry_prec prec, int32_t reorth, const double* b_dev,
                            int32_t k, double* x_dev, double* alphas, double* betas, double* z2, double* psi2,
                            double* pl, double* grad, double* psi_dev);

/* Parametric-bootstrap MSE of the kriging prediction of the latent field at
 * grid cells (Sec. 3.5, Eq. bootstrap_uq), theta and beta known: replicate b
 * draws x_b on the n1 x n2 grid of the last kry_set_mask with the
 * circulant-embedding sampler (as kry_sample, white noise
 * xi_dev + b * 2 * M1 * M2), forms r_b = A x_b + tau eps_b (eps_dev + b * p:
 * p standard normals), predicts x_hat_b = sigma^2 Sigma A^T K^-1 r_b at every
 * cell (CG on the nrep right-hand sides together, opts->prec / rtol / maxit;
 * FP64 covariance map) and writes var_dev[t] = (1/nrep) sum_b
 * (x_b(c_t) - x_hat_b(c_t))^2 for the flat row-major cells c_t of
 * cells_dev[ncell] (int64).  It estimates the simple-kriging variance; the MSE
 * of y at a cell adds tau^2.  M1, M2 as for kry_sample (kry_sample_size gives
 * the smallest usable torus).  The caller owns every buffer (device); the
 * library keeps 2 nrep (n1 n2 + p) doubles of scratch in the context.
 * Errors: KRY_EINVAL for bad arguments or a target cell outside the grid (its
 * variance is NaN); KRY_ENOCONV when some replicate's CG missed rtol (the
 * variances are still written).  Synchronises the stream. */
kry_status kry_bootstrap_var(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts, int32_t nrep, int32_t M1,
                             int32_t M2, const double* xi_dev, const double* eps_dev, const int64_t* cells_dev,
                             int64_t ncell, double* var_dev);

/* BCCB approximation of the log-determinant of the latent covariance
 * Sigma(theta) on the n1 x n2 grid of the last kry_set_mask (Sec. 3.3,
 * "Log-determinant approximation"), and of its derivative with respect to the
 * range (Appendix A, Eq. circ_diag and Eq. trace_approx):
 *   *logdet = (n1 n2 / (M1 M2)) sum_k log D1_k,
 *   *dlogdet_drange = (n1 n2 / (M1 M2)) sum_k D2_k / D1_k,
 * D1 and D2 the eigenvalues (2-D FFT of the first row) of the block-circulant
 * extensions of Sigma and d Sigma / d(range) on the matvec's M1 x M2 torus
 * (M_d the smallest power of two >= 2 n_d; the paper's formula uses a
 * (2 n_d - 1)-point extension and its first n1 x n2 frequencies, a reading
 * this build does not take because that length is not a power of two).
 * sigma2, range, nu and anisotropy come from cov; its nugget tau2 is not part
 * of Sigma and is ignored.  Eigenvalues below 2^-52 max D1 are reset to that
 * value before the log (the Sec. 3.6 recourse) and add no derivative term.
 * FP64 throughout.  dlogdet_drange may be NULL (no derivative computed).
 * Errors: KRY_EINVAL without a mask or for bad cov; KRY_ENAN for a non-finite
 * result.  Synchronises the stream. */
kry_status kry_bccb_logdet(kry_ctx* ctx, const kry_cov* cov, double* logdet, double* dlogdet_drange);

/* Smallest torus for kry_sample: starting from M_d = smallest power of two
 * >= 2 n_d, doubles both sides (at most 3 times, never past 8192) until
 * min(Lambda) >= -1e-10 max(Lambda).  Returns KRY_ENOTPSD with the largest
 * size tried if none qualifies.  Synchronises the stream. */
kry_status kry_sample_size(kry_ctx* ctx, const kry_cov* cov, int32_t* M1, int32_t* M2);

/* ---- Continuous-batching server (no counterpart in the paper; it serves many
 * independent likelihood or kriging requests on one GPU).
 *
 * A server runs nslots worker threads, each with its own CUDA stream and
 * context, so requests in different slots overlap on the device.  Requests
 * wait in one queue; a free slot admits the first queued request whose
 * estimated device footprint fits in what mem_budget_bytes has left (smaller
 * requests may pass a large one that does not fit yet; an idle slot gives its
 * cached buffers back when a queued request cannot be admitted).  All request
 * buffers are host memory owned by the caller and must stay valid until
 * kry_server_wait returns for the ticket.  A request is computed exactly as a
 * kry_profile_loglik (kind KRY_REQ_LOGLIK, one setting) or kry_krige (kind
 * KRY_REQ_KRIGE, means at the given target cells) call in a fresh context
 * with default launch schedules, so its result does not depend on what else
 * runs. */
typedef enum { KRY_REQ_LOGLIK = 0, KRY_REQ_KRIGE = 1 } kry_request_kind;

typedef struct {
    int32_t kind;                  /* kry_request_kind */
    int32_t n1, n2;                /* grid, cell sizes 1/n1 x 1/n2 */
    const uint8_t* mask;           /* n1*n2 bytes, row-major, nonzero = observed */
    const double* y;               /* p observations (row-major order of observed cells) */
    const double* X;               /* p x ncov covariates, column-major */
    int32_t ncov;
    kry_cov cov;
    kry_opts opts;
    double* loglik;                /* out (LOGLIK): profile log-likelihood */
    double* logdet;                /* out (LOGLIK, may be NULL): log det K estimate */
    double* beta;                  /* out (may be NULL): ncov GLS coefficients */
    const int64_t* target_cells;   /* KRIGE: the N - p unobserved cells, row-major indices */
    const double* target_X;        /* KRIGE: (N - p) x ncov covariates at those cells, column-major */
    double* mean;                  /* out (KRIGE): N - p kriging means */
} kry_request;

typedef struct kry_server kry_server;

kry_status kry_server_create(kry_server** server, int device, int32_t nslots, int64_t mem_budget_bytes);
/* Queue a request (returns at once).  KRY_ENOMEM if it can never fit the budget. */
kry_status kry_server_submit(kry_server* server, const kry_request* req, uint64_t* ticket);
/* Wait at most timeout_s seconds for a ticket (KRY_ETIMEOUT if it has not
 * finished).  On completion reports the request's own status, its latency
 * from submission to completion in ms, the slot that ran it and (err_buf of
 * err_len bytes, may be NULL) the request's error message; the ticket is then
 * retired. */
kry_status kry_server_wait(kry_server* server, uint64_t ticket, double timeout_s, kry_status* req_status,
                           double* latency_ms, int32_t* slot, char* err_buf, int32_t err_len);
/* Requests queued and not yet admitted. */
int64_t kry_server_queued(kry_server* server);
/* Stops the workers after their current request; queued requests are dropped. */
void kry_server_destroy(kry_server* server);

/* Schedule autotuner (no counterpart in the paper; the paper names no GPU
 * schedule).  Times every feasible launch schedule of the covariance matvec on
 * embedding e for batches of nvec vectors -- rows per block of the row passes,
 * columns per block (= slab tile width) of the column pass, and complex pairs
 * per batch (all, or chunks whose FFT intermediate fits ~32/64 MB of L2) --
 * and keeps the fastest for (M1, M2, precision, batch-size bucket) in ctx;
 * every later matvec, log-det, solve and likelihood on ctx with that shape
 * uses it.  Reports the best time per call (ms) and the chosen schedule
 * (host pointers, each may be NULL).  Allocates and frees two test buffers
 * of nvec * p values.  Synchronises the stream. */
kry_status kry_autotune(kry_ctx* ctx, const kry_embed* e, int32_t nvec, double* best_ms,
                        int32_t* rows_per_block, int32_t* cols_per_block, int32_t* pairs_per_batch);
/* Set that schedule explicitly (0 = library default for each field). */
kry_status kry_set_schedule(kry_ctx* ctx, const kry_embed* e, int32_t nvec, int32_t rows_per_block,
                            int32_t cols_per_block, int32_t pairs_per_batch);

/* Diagnostics (no counterpart in the paper).  kry_profile_enable(ctx, 1)
 * starts timing every covariance matvec issued on ctx (the three FFT passes
 * of one call, CUDA events on the context stream) and clears earlier records;
 * 0 stops.  kry_profile_read sums the records of one precision (KRY_F32 or
 * KRY_F64): number of matvec calls, real vectors transformed, and device
 * milliseconds.  Both synchronise the stream. */
kry_status kry_profile_enable(kry_ctx* ctx, int on);
kry_status kry_profile_read(kry_ctx* ctx, int32_t prec, int64_t* calls, int64_t* vectors, double* total_ms);

/* Number of kernels this library has launched in this process. */
uint64_t kry_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* KRY_H */
