// Circulant embedding of the BTTB covariance and its eigenvalues (Sec. 3.3:
// the block-circulant matrix built from one row of Sigma; Appendix A,
// Eq. circ_diag: a BCCB matrix is diagonalised by the 2-D Fourier matrix),
// and Gaussian-process sampling on the same embedding (Sec. 3.5 bootstrap;
// Sec. 3.6 caveat on negative eigenvalues).
//
// The first row c of the embedding lives on an M1 x M2 torus, M_d the
// smallest power of two >= 2 n_d.  A torus index j maps to the lag of its
// minimal image (j, or j - M when j > M/2); at j = M/2 the two images +-M/2
// are averaged, which keeps c symmetric under j -> -j (and Lambda real) for
// anisotropic covariances too.  Lambda = FFT2(c) in FP64.
#include <algorithm>
#include <cfloat>

#include "fft.cuh"
#include "kry_internal.cuh"
#include "matern.cuh"
#include "mvspec.cuh"

namespace kry {

// ------------------------------------------------------------------ twiddles

__global__ void k_twiddles(double2* tw64, float2* tw32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= KRY_TWN) return;
    double s, c;
    sincospi(-2.0 * (double)k / (double)KRY_TWN, &s, &c);
    tw64[k] = make_double2(c, s);
    tw32[k] = make_float2((float)c, (float)s);
}

void init_twiddles(kry_ctx* ctx) {
    ctx->tw64.ensure(KRY_TWN * sizeof(double2));
    ctx->tw32.ensure(KRY_TWN * sizeof(float2));
    k_twiddles<<<(KRY_TWN + 255) / 256, 256, 0, ctx->stream>>>(ctx->tw64.as<double2>(), ctx->tw32.as<float2>());
    KRY_CHECK_LAUNCH();
    ctx->twt32.ensure((size_t)kspec::TWT_ROWS * 16 * sizeof(float2));
    kspec::fill_stage_twiddles(ctx->twt32.as<float2>(), ctx->stream);
}

// ------------------------------------------------------------------ lag covariance

struct CovDev {
    double sigma2, inv_range, nu, ca, sa, ratio, dx1, dx2;
};

__device__ __forceinline__ double cov_at(const CovDev& p, double l1, double l2) {
    const double r = kry_scaled_dist(l1 * p.dx1, l2 * p.dx2, p.ca, p.sa, p.ratio, p.inv_range);
    return p.sigma2 * kry_matern(r, p.nu);
}

// d/d(range) of sigma^2 rho(d / range): with r = d / range, dr / d(range) = -r / range.
__device__ __forceinline__ double cov_drange_at(const CovDev& p, double l1, double l2) {
    const double r = kry_scaled_dist(l1 * p.dx1, l2 * p.dx2, p.ca, p.sa, p.ratio, p.inv_range);
    if (r <= 0.0) return 0.0;
    return p.sigma2 * kry_matern_dr(r, p.nu) * (-r * p.inv_range);
}

template <bool DRANGE>
__device__ __forceinline__ double lag_entry(const CovDev& p, double l1, double l2) {
    return DRANGE ? cov_drange_at(p, l1, l2) : cov_at(p, l1, l2);
}

// First row of the block-circulant extension of the covariance (DRANGE: of
// its range derivative) on the M1 x M2 torus.
template <bool DRANGE = false>
__global__ void k_lag_cov(double* __restrict__ c, int M1, int M2, CovDev p) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M1 * M2) return;
    const int j1 = (int)(idx / M2);
    const int j2 = (int)(idx - (int64_t)j1 * M2);
    const int a1 = (2 * j1 <= M1) ? j1 : j1 - M1;
    const int b1 = (2 * j1 < M1) ? j1 : j1 - M1;
    const int a2 = (2 * j2 <= M2) ? j2 : j2 - M2;
    const int b2 = (2 * j2 < M2) ? j2 : j2 - M2;
    double v;
    if (a1 == b1 && a2 == b2) {
        v = lag_entry<DRANGE>(p, a1, a2);
    } else if (a1 == b1) {
        v = 0.5 * (lag_entry<DRANGE>(p, a1, a2) + lag_entry<DRANGE>(p, a1, b2));
    } else if (a2 == b2) {
        v = 0.5 * (lag_entry<DRANGE>(p, a1, a2) + lag_entry<DRANGE>(p, b1, a2));
    } else {
        v = 0.25 * (lag_entry<DRANGE>(p, a1, a2) + lag_entry<DRANGE>(p, a1, b2) + lag_entry<DRANGE>(p, b1, a2) +
                    lag_entry<DRANGE>(p, b1, b2));
    }
    c[idx] = v;
}

// ------------------------------------------------------------------ full FP64 2-D FFT

// Row transforms over all M1 rows (length M2), G rows per CTA.
// IN 0: real input rows (c);  IN 1: sqrt(max(lam, 0) * scale) * (xi_re + i xi_im).
template <int EPT, int G, int IN>
__global__ void __launch_bounds__(EPT >= 16 ? 512 : 1024) k_rows_full(const double* __restrict__ rin, const double* __restrict__ xi,
                                                    double scale, double2* __restrict__ z, int M1, int M2,
                                                    const double2* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int L = M2, stride = L + 1, LT = L / EPT;
    const int g = threadIdx.x / LT, tl = threadIdx.x - g * LT;
    const int row = blockIdx.x * G + g;
    double2* rb = buf + g * stride;
    if (row < M1) {
        const int64_t off = (int64_t)row * M2;
        for (int k = tl; k < L; k += LT) {
            if (IN == 0) {
                rb[k] = make_double2(rin[off + k], 0.0);
            } else {
                const double a = sqrt(fmax(rin[off + k], 0.0) * scale);
                rb[k] = make_double2(a * xi[off + k], a * xi[(int64_t)M1 * M2 + off + k]);
            }
        }
    } else {
        for (int k = tl; k < L; k += LT) rb[k] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    fft_smem<double2, false, EPT>(rb, L, tl, tw);
    if (row < M1) {
        const int64_t off = (int64_t)row * M2;
        for (int k = tl; k < L; k += LT) z[off + k] = rb[k];
    }
}

// Column transforms (length M1) of CC columns per CTA; writes the real part.
// OUT 0: lam[k1][j] for every column;  OUT 1: out[i][j] for i < n1, j < n2.
template <int EPT, int CC, int OUT>
__global__ void __launch_bounds__(EPT >= 16 ? 512 : 1024) k_cols_full(const double2* __restrict__ z, double* __restrict__ out, int M1,
                                                    int M2, int n1, int n2, const double2* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* buf = reinterpret_cast<double2*>(smem_raw);
    const int L = M1, stride = L + 1, LT = L / EPT;
    const int g = threadIdx.x / LT, tl = threadIdx.x - g * LT;
    const int j0 = blockIdx.x * CC;
    for (int e = threadIdx.x; e < L * CC; e += blockDim.x) {
        const int k = e / CC, c = e - k * CC;
        buf[c * stride + k] = z[(int64_t)k * M2 + j0 + c];
    }
    __syncthreads();
    double2* cb = buf + g * stride;
    fft_smem<double2, false, EPT>(cb, L, tl, tw);
    if (OUT == 0) {
        for (int e = threadIdx.x; e < L * CC; e += blockDim.x) {
            const int k = e / CC, c = e - k * CC;
            out[(int64_t)k * M2 + j0 + c] = buf[c * stride + k].x;
        }
    } else {
        for (int e = threadIdx.x; e < n1 * CC; e += blockDim.x) {
            const int k = e / CC, c = e - k * CC;
            if (j0 + c < n2) out[(int64_t)k * n2 + j0 + c] = buf[c * stride + k].x;
        }
    }
}

static int pick_group(int L, int ept, size_t bytes_per_elem, size_t lim) {
    int g = 1;
    while (g < 8 && (size_t)(2 * g) * (L + 1) * bytes_per_elem <= lim && 2 * g * (L / ept) <= 256) g *= 2;
    return g;
}

template <int IN>
static void launch_rows_full(kry_ctx* ctx, const double* rin, const double* xi, double scale, double2* z, int M1,
                             int M2) {
    const int ept = (M2 >= 8192) ? 16 : 8;
    const int G = pick_group(M2, ept, sizeof(double2), ctx->max_smem_optin - 1024);
    const int thr = G * (M2 / ept);
    const size_t sm = (size_t)G * (M2 + 1) * sizeof(double2);
    const int nb = (M1 + G - 1) / G;
    const double2* tw = ctx->tw64.as<double2>();
#define KRY_ROWS(E, GG)                                                                     \
    do {                                                                                    \
        auto k = k_rows_full<E, GG, IN>;                                                    \
        KRY_ALLOW_MAX_SMEM(k); \
        k<<<nb, thr, sm, ctx->stream>>>(rin, xi, scale, z, M1, M2, tw);                     \
    } while (0)
    if (ept == 8) {
        if (G == 1) KRY_ROWS(8, 1); else if (G == 2) KRY_ROWS(8, 2); else if (G == 4) KRY_ROWS(8, 4); else KRY_ROWS(8, 8);
    } else {
        if (G == 1) KRY_ROWS(16, 1); else if (G == 2) KRY_ROWS(16, 2); else if (G == 4) KRY_ROWS(16, 4); else KRY_ROWS(16, 8);
    }
#undef KRY_ROWS
    KRY_CHECK_LAUNCH();
}

template <int OUT>
static void launch_cols_full(kry_ctx* ctx, const double2* z, double* out, int M1, int M2, int n1, int n2) {
    const int ept = (M1 >= 8192) ? 16 : 8;
    int C = pick_group(M1, ept, sizeof(double2), ctx->max_smem_optin - 1024);
    while (C > 1 && M2 % C) C /= 2;
    const int thr = C * (M1 / ept);
    const size_t sm = (size_t)C * (M1 + 1) * sizeof(double2);
    int nb = M2 / C;
    if (OUT == 1) nb = (n2 + C - 1) / C;
    const double2* tw = ctx->tw64.as<double2>();
#define KRY_COLS(E, CCV)                                                                    \
    do {                                                                                    \
        auto k = k_cols_full<E, CCV, OUT>;                                                  \
        KRY_ALLOW_MAX_SMEM(k); \
        k<<<nb, thr, sm, ctx->stream>>>(z, out, M1, M2, n1, n2, tw);                        \
    } while (0)
    if (ept == 8) {
        if (C == 1) KRY_COLS(8, 1); else if (C == 2) KRY_COLS(8, 2); else if (C == 4) KRY_COLS(8, 4); else KRY_COLS(8, 8);
    } else {
        if (C == 1) KRY_COLS(16, 1); else if (C == 2) KRY_COLS(16, 2); else if (C == 4) KRY_COLS(16, 4); else KRY_COLS(16, 8);
    }
#undef KRY_COLS
    KRY_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ min / max

__global__ void k_minmax(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
    __shared__ double smin[32], smax[32];
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, smin[w]);
            hi = fmax(hi, smax[w]);
        }
        lo = fmin(lo, smin[0]);
        hi = fmax(hi, smax[0]);
        part[2 * blockIdx.x] = lo;
        part[2 * blockIdx.x + 1] = hi;
    }
}

__global__ void k_minmax_final(double* part, int nb) {
    double lo = DBL_MAX, hi = -DBL_MAX;
    for (int b = 0; b < nb; ++b) {
        lo = fmin(lo, part[2 * b]);
        hi = fmax(hi, part[2 * b + 1]);
    }
    part[0] = lo;
    part[1] = hi;
}

static CovDev cov_dev(const kry_cov& cov, double dx1, double dx2) {
    CovDev p;
    p.sigma2 = cov.sigma2;
    p.inv_range = 1.0 / cov.range;
    p.nu = cov.nu;
    p.ca = cos(cov.aniso_angle);
    p.sa = sin(cov.aniso_angle);
    p.ratio = cov.aniso_ratio;
    p.dx1 = dx1;
    p.dx2 = dx2;
    return p;
}

void compute_eigs(kry_ctx* ctx, const kry_cov& cov, int n1, int n2, double dx1, double dx2, int M1, int M2,
                  double* lam_min, double* lam_max) {
    const int64_t MM = (int64_t)M1 * M2;
    ctx->eig_c.ensure(MM * sizeof(double));
    ctx->eig_z.ensure(MM * sizeof(double2));
    double* c = ctx->eig_c.as<double>();
    double2* z = ctx->eig_z.as<double2>();
    (void)n1;
    (void)n2;
    k_lag_cov<<<(unsigned)((MM + 255) / 256), 256, 0, ctx->stream>>>(c, M1, M2, cov_dev(cov, dx1, dx2));
    KRY_CHECK_LAUNCH();
    launch_rows_full<0>(ctx, c, nullptr, 0.0, z, M1, M2);
    launch_cols_full<0>(ctx, z, c, M1, M2, 0, 0);   // Lambda (real part) back into c
    const int nb = 256;
    ctx->red.ensure(2 * nb * sizeof(double));
    k_minmax<<<nb, 256, 0, ctx->stream>>>(c, MM, ctx->red.as<double>());
    KRY_CHECK_LAUNCH();
    k_minmax_final<<<1, 1, 0, ctx->stream>>>(ctx->red.as<double>(), nb);
    KRY_CHECK_LAUNCH();
    KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned, ctx->red.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    *lam_min = ctx->host_pinned[0];
    *lam_max = ctx->host_pinned[1];
}

// Eigenvalues of (S + tau2 I)^-1 from those of the embedding S (in
// ctx->eig_c): 1 / (max(Lambda, 0) + tau2).  Negative embedding eigenvalues
// are reset to zero first (Sec. 3.6 caveat) so that the inverse stays
// positive definite.
__global__ void k_invert_eigs(double* __restrict__ c, int64_t MM, double tau2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MM; i += (int64_t)gridDim.x * blockDim.x)
        c[i] = 1.0 / (fmax(c[i], 0.0) + tau2);
}

void invert_eigs(kry_ctx* ctx, int M1, int M2, double tau2) {
    const int64_t MM = (int64_t)M1 * M2;
    k_invert_eigs<<<(unsigned)std::min<int64_t>((MM + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        ctx->eig_c.as<double>(), MM, tau2);
    KRY_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ BCCB log-determinant
//
// Sec. 3.3's approximation log det Sigma ~ sum log D1 and its range
// derivative dL ~ sum D2 / D1 (Appendix A, Eq. circ_diag and Eq.
// trace_approx), D1 and D2 the eigenvalues of the block-circulant extensions
// of Sigma and d Sigma / d(range).  Reading: the matvec's power-of-two
// M1 x M2 torus, all frequencies, scaled by n1 n2 / (M1 M2) (the paper's
// (2n - 1)-point extension is not a power of two).  Eigenvalues below
// eps * max D1 are reset to that value (Sec. 3.6) and add no derivative term.

// Per-block sums of log(max(D1, floor)) and, where D1 > floor, D2 / D1.
__global__ void k_bccb_partials(const double* __restrict__ d1, const double* __restrict__ d2, int64_t n,
                                double floor_v, double* __restrict__ part) {
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double l = d1[i];
        const bool keep = l > floor_v;
        a += log(keep ? l : floor_v);
        if (keep && d2) b += d2[i] / l;
    }
    __shared__ double sa[256], sb[256];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sa[threadIdx.x] += sa[threadIdx.x + o];
            sb[threadIdx.x] += sb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sa[0];
        part[2 * blockIdx.x + 1] = sb[0];
    }
}

__global__ void k_bccb_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    out[0] = a;
    out[1] = b;
}

void bccb_logdet(kry_ctx* ctx, const kry_cov& cov, bool deriv, double* logdet, double* dlogdet) {
    const int n1 = ctx->n1, n2 = ctx->n2;
    int M1 = 1, M2 = 1;
    while (M1 < 2 * n1) M1 <<= 1;
    while (M2 < 2 * n2) M2 <<= 1;
    const int64_t MM = (int64_t)M1 * M2;
    double lo, hi;
    compute_eigs(ctx, cov, n1, n2, ctx->dx1, ctx->dx2, M1, M2, &lo, &hi);   // D1 in eig_c
    double* d1 = ctx->eig_c.as<double>();
    double* d2 = nullptr;
    if (deriv) {
        ctx->eig_d.ensure(MM * sizeof(double));
        d2 = ctx->eig_d.as<double>();
        k_lag_cov<true><<<(unsigned)((MM + 255) / 256), 256, 0, ctx->stream>>>(d2, M1, M2,
                                                                            cov_dev(cov, ctx->dx1, ctx->dx2));
        KRY_CHECK_LAUNCH();
        double2* z = ctx->eig_z.as<double2>();
        launch_rows_full<0>(ctx, d2, nullptr, 0.0, z, M1, M2);
        launch_cols_full<0>(ctx, z, d2, M1, M2, 0, 0);   // D2 (real part) back into d2
    }
    const int nb = 256;
    ctx->red.ensure((2 * nb + 2) * sizeof(double));
    double* part = ctx->red.as<double>();
    k_bccb_partials<<<nb, 256, 0, ctx->stream>>>(d1, d2, MM, 2.220446049250313e-16 * hi, part);
    KRY_CHECK_LAUNCH();
    k_bccb_final<<<1, 1, 0, ctx->stream>>>(part, nb, part + 2 * nb);
    KRY_CHECK_LAUNCH();
    KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned, part + 2 * nb, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                             ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    const double scale = (double)n1 * (double)n2 / (double)MM;
    *logdet = scale * ctx->host_pinned[0];
    if (dlogdet) *dlogdet = scale * ctx->host_pinned[1];
}

// lamT[j][k] = lam[k][j] * scale (FP64 and optionally FP32), 32 x 32 tiles.
// With t32p != NULL also the column-permuted FP32 copy: row k = t + m M1/16 of
// column j goes to t32p[j M1 + 16 t + m].
__global__ void k_transpose_scale(const double* __restrict__ lam, int M1, int M2, double scale,
                                  double* __restrict__ t64, float* __restrict__ t32, float* __restrict__ t32p) {
    const int lt = M1 >> 4;
    __shared__ double tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int k = by + r, j = bx + threadIdx.x;
        if (k < M1 && j < M2) tile[r][threadIdx.x] = lam[(int64_t)k * M2 + j];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = bx + r, k = by + threadIdx.x;
        if (k < M1 && j < M2) {
            const double v = tile[threadIdx.x][r] * scale;
            t64[(int64_t)j * M1 + k] = v;
            if (t32) t32[(int64_t)j * M1 + k] = (float)v;
            if (t32p) t32p[(int64_t)j * M1 + (k % lt) * 16 + k / lt] = (float)v;
        }
    }
}

// Store the eigenvalues in ctx->eig_c as setting `slot` of embedding e.
void store_embedding(kry_ctx* ctx, kry_embed* e, int slot) {
    dim3 grid((e->M2 + 31) / 32, (e->M1 + 31) / 32), blk(32, 8);
    const int64_t off = (int64_t)slot * e->M1 * e->M2;
    k_transpose_scale<<<grid, blk, 0, ctx->stream>>>(ctx->eig_c.as<double>(), e->M1, e->M2,
                                                     1.0 / ((double)e->M1 * (double)e->M2), e->lam64T + off,
                                                     e->lam32T ? e->lam32T + off : nullptr,
                                                     e->lam32P ? e->lam32P + off : nullptr);
    KRY_CHECK_LAUNCH();
}

// Replace the eigenvalues of FP64 embedding e (one setting, e's grid) by those
// of the circulant extension of d Sigma / d(range) for cov, so that matvecs
// with e apply the range derivative of the covariance (Appendix A, dSigma).
void drange_embedding(kry_ctx* ctx, const kry_cov& cov, kry_embed* e) {
    const int M1 = e->M1, M2 = e->M2;
    const int64_t MM = (int64_t)M1 * M2;
    ctx->eig_c.ensure(MM * sizeof(double));
    ctx->eig_z.ensure(MM * sizeof(double2));
    double* c = ctx->eig_c.as<double>();
    double2* z = ctx->eig_z.as<double2>();
    k_lag_cov<true><<<(unsigned)((MM + 255) / 256), 256, 0, ctx->stream>>>(c, M1, M2,
                                                                        cov_dev(cov, ctx->dx1, ctx->dx2));
    KRY_CHECK_LAUNCH();
    launch_rows_full<0>(ctx, c, nullptr, 0.0, z, M1, M2);
    launch_cols_full<0>(ctx, z, c, M1, M2, 0, 0);
    store_embedding(ctx, e, 0);
}


void sample_field(kry_ctx* ctx, const kry_cov& cov, int M1, int M2, const double* xi, double* out) {
    double lo, hi;
    compute_eigs(ctx, cov, ctx->n1, ctx->n2, ctx->dx1, ctx->dx2, M1, M2, &lo, &hi);
    double2* z = ctx->eig_z.as<double2>();
    launch_rows_full<1>(ctx, ctx->eig_c.as<double>(), xi, 1.0 / ((double)M1 * (double)M2), z, M1, M2);
    launch_cols_full<1>(ctx, z, out, M1, M2, ctx->n1, ctx->n2);
}

}  // namespace kry
