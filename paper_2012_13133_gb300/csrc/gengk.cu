// genHyBR for the latent field (Sec. 3.2): generalized Golub-Kahan
// bidiagonalization (Alg. 1) with A = the observed-cell selection, Sigma =
// the correlation matrix (sigma^2 = 1) applied on the whole grid by the
// circulant-embedding matvec, R = tau^2 I; the projected Tikhonov problem
// (B_k^T B_k + I / sigma^2) z = B_k^T beta1 e1; x_k* = Sigma V_k z_k (Eq.
// xhat_est); and the approximate profile log-likelihood of Eq. prof_lik with
// the BCCB log-det of Sec. 3.3.
//
// Reading of the garbled beta_{i+1} step of Alg. 1: beta_{i+1} =
// ||A Sigma v_i - alpha_i u_i||_2 / tau, as beta_1 = ||b||_2 / tau, which is
// what U^T U = tau^2 I (Eq. exact_arith) requires.  No reorthogonalisation
// (the paper runs without it).
//
// Two precisions: FP64 throughout, or FP32 Krylov vectors (u_i, v_i, Sigma v_i
// and the whole-grid FP32 matvec) with every norm, inner product and scalar
// of the recurrence accumulated and kept in FP64.
//
// The whole-grid matvec reuses the passes of the observed-cell matvec with
// the row/column index lists of a full mask swapped in for the duration of
// each call; pass C's fused dot product gives w^T Sigma w, the squared
// Sigma-norm of Alg. 1.
#include <math.h>

#include <algorithm>
#include <vector>

#include "gengk.cuh"
#include "kry_internal.cuh"

namespace kry {

template <typename T>
void matvec_ex(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
               int64_t ld_out, int nvec, double* dots, int nds, int vpt = 0, const int* skip = nullptr);
int matvec_num_partials(kry_ctx* ctx, const kry_embed* e, bool dbl, int nvec);

namespace {

__global__ void k_full_index(int* __restrict__ rowptr, int* __restrict__ colidx, int n1, int n2) {
    const int64_t N = (int64_t)n1 * n2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        colidx[i] = (int)(i % n2);
        if (i % n2 == 0) rowptr[i / n2] = (int)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n1] = (int)N;
}

// Swaps the full-grid index lists into the context for one scope.
struct FullGrid {
    kry_ctx* ctx;
    int64_t p_saved;
    explicit FullGrid(kry_ctx* c) : ctx(c), p_saved(c->p) {
        std::swap(ctx->rowptr, ctx->rowptr_full);
        std::swap(ctx->colidx, ctx->colidx_full);
        ctx->p = (int64_t)ctx->n1 * ctx->n2;
    }
    ~FullGrid() {
        std::swap(ctx->rowptr, ctx->rowptr_full);
        std::swap(ctx->colidx, ctx->colidx_full);
        ctx->p = p_saved;
    }
};

// Per-block partial sums of x[i]^2 in FP64 (fixed order within a block).
template <typename T>
__global__ void k_sq_partials(const T* __restrict__ x, int64_t n, double* __restrict__ part) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s += v * v;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// t[q] = sv[cell q] - alpha u[q]
template <typename TS, typename TU, typename TO>
__global__ void k_gk_gather(const TS* __restrict__ sv, const int* __restrict__ cellidx, const TU* __restrict__ u,
                            double alpha, TO* __restrict__ t, int64_t p) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p; q += (int64_t)gridDim.x * blockDim.x)
        t[q] = (TO)((double)sv[cellidx[q]] - alpha * (double)u[q]);
}

template <typename TI, typename TO>
__global__ void k_scale_copy(const TI* __restrict__ x, double s, TO* __restrict__ y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (TO)(s * (double)x[i]);
}

// w = -beta v (whole grid), then w[cell q] += u[q] / tau^2 (cells are distinct)
template <typename T>
__global__ void k_gk_fill(const T* __restrict__ v, double beta, T* __restrict__ w, int64_t N) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = (T)(-beta * (double)v[i]);
}
template <typename T>
__global__ void k_gk_scatter_add(const T* __restrict__ u, const int* __restrict__ cellidx, double inv_tau2,
                                 T* __restrict__ w, int64_t p) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = cellidx[q];
        w[c] = (T)((double)w[c] + inv_tau2 * (double)u[q]);
    }
}

// out[i] = sum_j z[j] V[j][i]  (j < k, fixed order, FP64 accumulation)
template <typename T>
__global__ void k_gk_combine(const T* __restrict__ V, const double* __restrict__ z, int k, int64_t N,
                             T* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += z[j] * (double)V[(int64_t)j * N + i];
        out[i] = (T)s;
    }
}

// Reorthogonalisation (optional; the paper runs Alg. 1 without it): the new u
// against U (Euclidean, U^T U = tau^2 I) and the new w against V (Sigma inner
// product, V^T Sigma V = I, through the stored Sigma V), two classical
// Gram-Schmidt passes each.
//   part[j][b] = block b's FP64 partial of A_j^T x (j < m; A_j = A + j stride)
template <typename T>
__global__ void k_mdot(const T* __restrict__ A, int64_t stride, int m, const T* __restrict__ x, int64_t n,
                       double* __restrict__ part) {
    __shared__ double sh[256];
    for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            s += (double)A[(int64_t)j * stride + i] * (double)x[i];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = sh[0];
        __syncthreads();
    }
}

//   c[j] = scale * sum_b part[j][b]  (one thread per j, fixed order)
__global__ void k_mdot_finish(const double* __restrict__ part, int nb, int m, double scale, double* __restrict__ c) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)j * nb + b];
    c[j] = scale * s;
}

//   x -= sum_j c[j] B_j  (FP64 accumulation, j in a fixed order)
template <typename T>
__global__ void k_maxpy(const T* __restrict__ B, int64_t stride, int m, const double* __restrict__ c,
                        T* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < m; ++j) s += c[j] * (double)B[(int64_t)j * stride + i];
        x[i] = (T)((double)x[i] - s);
    }
}

const int NB = 256;
const int NBR = 128;   // blocks of k_mdot

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

template <typename T>
double sum_sq(kry_ctx* ctx, const T* x, int64_t n, double* part) {
    k_sq_partials<T><<<NB, 256, 0, ctx->stream>>>(x, n, part);
    KRY_CHECK_LAUNCH();
    KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned, part, NB * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (int b = 0; b < NB; ++b) s += ctx->host_pinned[b];
    return s;
}

// sw = Sigma w on the whole grid; returns w^T Sigma w.
template <typename T>
double sigma_full(kry_ctx* ctx, const kry_embed* e, const T* w, T* sw, double* dots, int nds) {
    {
        FullGrid fg(ctx);
        const int64_t N = ctx->p;
        matvec_ex<T>(ctx, e, w, N, nullptr, sw, N, 1, dots, nds);
    }
    KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned, dots, nds * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (int b = 0; b < nds; ++b) s += ctx->host_pinned[b];
    return s;
}

}  // namespace

namespace {

// x -= B (scale A^T x), twice (classical Gram-Schmidt, repeated), for the m
// columns of A and B (stride apart); part and c are FP64 scratch of m NBR and m.
template <typename T>
void project_out(kry_ctx* ctx, const T* A, const T* B, int64_t stride, int m, double scale, T* x, int64_t n,
                 double* part, double* c) {
    for (int pass = 0; pass < 2; ++pass) {
        k_mdot<T><<<NBR, 256, 0, ctx->stream>>>(A, stride, m, x, n, part);
        KRY_CHECK_LAUNCH();
        k_mdot_finish<<<(m + 127) / 128, 128, 0, ctx->stream>>>(part, NBR, m, scale, c);
        KRY_CHECK_LAUNCH();
        k_maxpy<T><<<grid_for(n), 256, 0, ctx->stream>>>(B, stride, m, c, x, n);
        KRY_CHECK_LAUNCH();
    }
}

template <typename T>
void genhybr_t(kry_ctx* ctx, const kry_cov& cov, const double* b, int k, bool reorth, double* x_out, double* alphas,
               double* betas, double* z2_out, double* psi2_out, double* pl_out, double* grad, double* psi_out) {
    constexpr kry_prec prec = sizeof(T) == 8 ? KRY_F64 : KRY_F32;
    const int n1 = ctx->n1, n2 = ctx->n2;
    const int64_t N = (int64_t)n1 * n2, p = ctx->p;
    KRY_REQUIRE(cov.tau2 > 0.0 && cov.sigma2 > 0.0, KRY_EINVAL, "genHyBR needs tau2 > 0 and sigma2 > 0");
    KRY_REQUIRE(N <= 4096 * 4096, KRY_EUNSUPPORTED, "grid too large for the whole-grid matvec");
    // whole-grid index lists (built once per mask)
    KRY_REQUIRE(k >= 1, KRY_EINVAL, "k must be >= 1");
    if (ctx->rowptr_full.p == nullptr || ctx->full_n1 != n1 || ctx->full_n2 != n2) {
        ctx->rowptr_full.ensure((size_t)(n1 + 1) * sizeof(int));
        ctx->colidx_full.ensure((size_t)N * sizeof(int));
        k_full_index<<<grid_for(N), 256, 0, ctx->stream>>>(ctx->rowptr_full.as<int>(), ctx->colidx_full.as<int>(), n1,
                                                           n2);
        KRY_CHECK_LAUNCH();
        ctx->full_n1 = n1;
        ctx->full_n2 = n2;
    }
    kry_cov corr = cov;
    corr.sigma2 = 1.0;
    corr.tau2 = 0.0;
    const double tau2 = cov.tau2, tau = sqrt(tau2);
    // scratch: partials, pass C partials (at most 8192), k coefficients, and
    // with reorthogonalisation its partials and coefficients (FP64); then V
    // [k+1][N], SV, W, X (whole grid), U [k+1][p], T (observed) and with
    // reorthogonalisation the Sigma v_j [k+1][N] as T
    int nds = 0;
    const size_t nr = reorth ? (size_t)(k + 1) * (NBR + 1) : 0;
    const size_t nd = 2 * NB + 8192 + (size_t)k + 1 + nr;
    ctx->gk.ensure(nd * sizeof(double) +
                   ((size_t)(k + 4) * N + (size_t)(k + 2) * p + (reorth ? (size_t)(k + 1) * N : 0)) * sizeof(T));
    double* part = ctx->gk.as<double>();
    double* dots = part + 2 * NB;
    double* zdev = dots + 8192;
    double* rpart = zdev + k + 1;
    double* rc = rpart + (reorth ? (size_t)(k + 1) * NBR : 0);
    T* V = reinterpret_cast<T*>(part + nd);
    T* SV = V + (size_t)(k + 1) * N;
    T* W = SV + N;
    T* X = W + N;
    T* U = X + N;
    T* Tt = U + (size_t)(k + 1) * p;
    T* SVh = reorth ? Tt + p : nullptr;
    // Sigma v_i: the history's slot i with reorthogonalisation, else one buffer
    auto svp = [&](int i) -> T* { return reorth ? SVh + (size_t)i * N : SV; };

    kry_embed* e = make_embed_internal(ctx, &corr, prec);
    try {
        {
            FullGrid fg(ctx);
            nds = matvec_num_partials(ctx, e, sizeof(T) == 8, 1);
        }
        KRY_REQUIRE(nds <= 4096, KRY_EUNSUPPORTED, "too many matvec partials");   // the pinned host buffer
        std::vector<double> al(k + 1, 0.0), be(k + 1, 0.0);
        // u_1 = b / beta_1, beta_1 = ||b|| / tau
        const double beta1 = sqrt(sum_sq<double>(ctx, b, p, part)) / tau;
        KRY_REQUIRE(beta1 > 0.0 && isfinite(beta1), KRY_EINVAL, "b must be finite and nonzero");
        be[0] = beta1;
        k_scale_copy<double, T><<<grid_for(p), 256, 0, ctx->stream>>>(b, 1.0 / beta1, U, p);
        KRY_CHECK_LAUNCH();
        // w = A^T u_1 / tau^2, alpha_1 = ||w||_Sigma, v_1 = w / alpha_1
        KRY_CUDA(cudaMemsetAsync(W, 0, N * sizeof(T), ctx->stream));
        k_gk_scatter_add<T><<<grid_for(p), 256, 0, ctx->stream>>>(U, ctx->cellidx.as<int>(), 1.0 / tau2, W, p);
        KRY_CHECK_LAUNCH();
        double a2 = sigma_full<T>(ctx, e, W, svp(0), dots, nds);
        KRY_REQUIRE(a2 > 0.0 && isfinite(a2), KRY_ENAN, "alpha_1 is not positive");
        al[0] = sqrt(a2);
        k_scale_copy<T, T><<<grid_for(N), 256, 0, ctx->stream>>>(W, 1.0 / al[0], V, N);
        KRY_CHECK_LAUNCH();
        k_scale_copy<T, T><<<grid_for(N), 256, 0, ctx->stream>>>(svp(0), 1.0 / al[0], svp(0), N);
        KRY_CHECK_LAUNCH();
        // A step whose beta or alpha falls below 1e-13 of the first one ends the bidiagonalization:
        // the Krylov space then holds the solution (an exact breakdown up to rounding), and the
        // projected problem uses the keff steps taken.
        int keff = k;
        for (int i = 0; i < k; ++i) {
            T* ui = U + (size_t)i * p;
            T* un = U + (size_t)(i + 1) * p;
            T* vi = V + (size_t)i * N;
            T* vn = V + (size_t)(i + 1) * N;
            // t = A Sigma v_i - alpha_i u_i, beta_{i+1} = ||t|| / tau, u_{i+1} = t / beta_{i+1}
            k_gk_gather<T, T, T><<<grid_for(p), 256, 0, ctx->stream>>>(svp(i), ctx->cellidx.as<int>(), ui, al[i], Tt,
                                                                      p);
            KRY_CHECK_LAUNCH();
            if (reorth) project_out<T>(ctx, U, U, p, i + 1, 1.0 / tau2, Tt, p, rpart, rc);
            be[i + 1] = sqrt(sum_sq<T>(ctx, Tt, p, part)) / tau;
            KRY_REQUIRE(isfinite(be[i + 1]), KRY_ENAN, "genGK: beta is NaN/Inf");
            if (!(be[i + 1] > 1e-13 * beta1)) {
                be[i + 1] = 0.0;
                keff = i + 1;
                break;
            }
            k_scale_copy<T, T><<<grid_for(p), 256, 0, ctx->stream>>>(Tt, 1.0 / be[i + 1], un, p);
            KRY_CHECK_LAUNCH();
            // w = A^T u_{i+1} / tau^2 - beta_{i+1} v_i, alpha_{i+1} = ||w||_Sigma
            k_gk_fill<T><<<grid_for(N), 256, 0, ctx->stream>>>(vi, be[i + 1], W, N);
            KRY_CHECK_LAUNCH();
            k_gk_scatter_add<T><<<grid_for(p), 256, 0, ctx->stream>>>(un, ctx->cellidx.as<int>(), 1.0 / tau2, W, p);
            KRY_CHECK_LAUNCH();
            if (reorth) project_out<T>(ctx, SVh, V, N, i + 1, 1.0, W, N, rpart, rc);
            a2 = sigma_full<T>(ctx, e, W, svp(i + 1), dots, nds);
            KRY_REQUIRE(isfinite(a2), KRY_ENAN, "genGK: alpha is NaN/Inf");
            if (!(a2 > 1e-26 * al[0] * al[0])) {
                keff = i + 1;
                break;
            }
            al[i + 1] = sqrt(a2);
            k_scale_copy<T, T><<<grid_for(N), 256, 0, ctx->stream>>>(W, 1.0 / al[i + 1], vn, N);
            KRY_CHECK_LAUNCH();
            k_scale_copy<T, T><<<grid_for(N), 256, 0, ctx->stream>>>(svp(i + 1), 1.0 / al[i + 1], svp(i + 1), N);
            KRY_CHECK_LAUNCH();
        }
        // projected Tikhonov problem: (B^T B + I / sigma^2) z = B^T beta1 e1, B (k+1) x k lower
        // bidiagonal; B^T B is tridiagonal: diag a_j^2 + b_{j+1}^2, off-diagonal a_{j+1} b_{j+1}
        const int kk = keff;
        std::vector<double> d(kk), o(kk > 0 ? kk - 1 : 0), z(kk, 0.0);
        for (int j = 0; j < kk; ++j) d[j] = al[j] * al[j] + be[j + 1] * be[j + 1] + 1.0 / cov.sigma2;
        for (int j = 0; j + 1 < kk; ++j) o[j] = al[j + 1] * be[j + 1];
        z[0] = al[0] * beta1;
        // symmetric tridiagonal solve (LDL^T without pivoting: the matrix is positive definite)
        std::vector<double> dd(d), zz(z);
        for (int j = 1; j < kk; ++j) {
            const double m = o[j - 1] / dd[j - 1];
            dd[j] -= m * o[j - 1];
            zz[j] -= m * zz[j - 1];
        }
        for (int j = kk - 1; j >= 0; --j) zz[j] = (zz[j] - (j + 1 < kk ? o[j] * zz[j + 1] : 0.0)) / dd[j];
        double z2 = 0.0;
        for (int j = 0; j < kk; ++j) z2 += zz[j] * zz[j];
        // x* = Sigma V_k z, psi = b - A x*
        KRY_CUDA(cudaMemcpyAsync(zdev, zz.data(), kk * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        k_gk_combine<T><<<grid_for(N), 256, 0, ctx->stream>>>(V, zdev, kk, N, W);
        KRY_CHECK_LAUNCH();
        sigma_full<T>(ctx, e, W, X, dots, nds);
        // x*[c] - b, formed in FP64 from the x* the caller receives
        k_gk_gather<T, double, T><<<grid_for(p), 256, 0, ctx->stream>>>(X, ctx->cellidx.as<int>(), b, 1.0, Tt, p);
        KRY_CHECK_LAUNCH();
        const double psi2 = sum_sq<T>(ctx, Tt, p, part);
        if (x_out) {
            k_scale_copy<T, double><<<grid_for(N), 256, 0, ctx->stream>>>(X, 1.0, x_out, N);
            KRY_CHECK_LAUNCH();
        }
        if (psi_out) {   // psi = b - A x* = -T
            k_scale_copy<T, double><<<grid_for(p), 256, 0, ctx->stream>>>(Tt, -1.0, psi_out, p);
            KRY_CHECK_LAUNCH();
        }
        // Appendix A, Eq. approx_grad: (V_k z_k)^T dSigma (V_k z_k), V_k z_k still in W
        double qdq = 0.0;
        if (grad) {
            drange_embedding(ctx, corr, e);   // e now applies dSigma
            qdq = sigma_full<T>(ctx, e, W, SV, dots, nds);
        }
        double ld = 0.0, dl = 0.0;
        bccb_logdet(ctx, corr, grad != nullptr, &ld, grad ? &dl : nullptr);
        const double pl = -0.5 * (double)p * log(tau2) - psi2 / (2.0 * tau2) - 0.5 * (double)N * log(cov.sigma2) -
                          0.5 * ld - z2 / (2.0 * cov.sigma2);
        if (grad) {
            const double lam2 = 1.0 / cov.sigma2, lame2 = 1.0 / tau2;
            grad[0] = (double)N / (2.0 * lam2) - 0.5 * z2;          // d pl / d lambda^2
            grad[1] = -0.5 * dl + 0.5 * lam2 * qdq;                 // d pl / d range
            grad[2] = (double)p / (2.0 * lame2) - 0.5 * psi2;       // d pl / d lambda_e^2
        }
        if (alphas) std::copy(al.begin(), al.end(), alphas);
        if (betas) std::copy(be.begin(), be.end(), betas);
        if (z2_out) *z2_out = z2;
        if (psi2_out) *psi2_out = psi2;
        if (pl_out) *pl_out = pl;
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        free_embed_internal(e);
        throw;
    }
    free_embed_internal(e);
}

}  // namespace

void genhybr_opt(kry_ctx* ctx, const kry_cov& cov, kry_prec prec, bool reorth, const double* b, int k, double* x_out,
                 double* alphas, double* betas, double* z2_out, double* psi2_out, double* pl_out, double* grad,
                 double* psi_out) {
    if (prec == KRY_F32)
        genhybr_t<float>(ctx, cov, b, k, reorth, x_out, alphas, betas, z2_out, psi2_out, pl_out, grad, psi_out);
    else
        genhybr_t<double>(ctx, cov, b, k, reorth, x_out, alphas, betas, z2_out, psi2_out, pl_out, grad, psi_out);
}

void genhybr(kry_ctx* ctx, const kry_cov& cov, kry_prec prec, const double* b, int k, double* x_out, double* alphas,
             double* betas, double* z2_out, double* psi2_out, double* pl_out, double* grad, double* psi_out) {
    genhybr_opt(ctx, cov, prec, false, b, k, x_out, alphas, betas, z2_out, psi2_out, pl_out, grad, psi_out);
}

}  // namespace kry
