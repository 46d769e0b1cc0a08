// C ABI of the Kryging library (declared in include/kry.h): argument
// validation, context and mask set-up, and the glue that sequences the
// kernels of embed.cu, matvec.cu and krylov.cu.  No computation of the hot
// path happens on the host beyond scalar bookkeeping.
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <vector>

#include "gengk.cuh"
#include "kry_internal.cuh"

// Interior share of the mask from which kry_opts.precond = 2 preconditions CG.
#define KRY_PRECOND_AUTO_INTERIOR 0.4

// FP32 Krylov iterates resolve K = sigma2 A Sigma A^T + tau2 I only while
// kappa u32 stays below one, u32 = 2^-24 and kappa = (max |Lambda| + tau2) /
// tau2 the bound on K's condition number that the embedding gives (every
// eigenvalue of K lies in [tau2, max |Lambda| + tau2]).  Measured on 1024^2
// and 2048^2 grids with half the cells observed (Matern 3/2, range 0.05, CG
// on [y, X] to 1e-6 with FP64 residual replacement, at most 20,000
// iterations): FP32 CG converged at kappa 3.3e6 on both grids (about 9,000
// iterations) and at 6.6e6 on 2048^2 (19,968), and stalled at 5.5e6 on
// 1024^2 (relative residual 1.6e-4) and 1.3e7 on 2048^2 (0.57).  The FP32
// log-det with partial reorthogonalisation stayed within 1.2e-5 of the FP64
// one throughout.  Above 4e6 (kappa u32 = 0.24), likelihood, kriging and
// bootstrap calls with prec = KRY_AUTO run that setting in FP64 instead of
// FP32 (counted by kry_promoted).
#define KRY_F32_KAPPA_MAX 4.0e6

namespace kry {
void store_embedding(kry_ctx* ctx, kry_embed* e, int slot);
void logdet_batched(kry_ctx* ctx, const kry_embed* e, int nprobe, int nsteps, uint64_t seed, bool reorth,
                    double* per_vec);
template <typename T>
void matvec_ex(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
               int64_t ld_out, int nvec, double* dots, int nds, int vpt = 0, const int* skip = nullptr);
void logdet(kry_ctx* ctx, const kry_embed* e, int nprobe, int nsteps, uint64_t seed, bool reorth, double* per_probe);
SolveInfo solve(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, double* X, int64_t ldx, int nrhs,
                double rtol, int maxit, int vpt = 0, const kry_embed* pre = nullptr);
GlsResult gls(kry_ctx* ctx, const double* V, const double* Z, int ncov, double logdet);
void resid_weights(kry_ctx* ctx, const double* Z, int ncov, const double* beta_dev, double* w);
void krige_launch_cells(kry_ctx* ctx, const double* grid, const int64_t* cells, int64_t ncell, const double* Xc,
                        int ncov, const double* beta_dev, double* mean, int* bad);
void krige_launch_sites(kry_ctx* ctx, const kry_cov& cov, const double* sites, int64_t nsite, const double* Xs,
                        int ncov, const double* beta_dev, const double* w, double* mean);
bool krige_variances(kry_ctx* ctx, const kry_embed* e, const int64_t* cells, int64_t ncell, double* var,
                     double rtol, int maxit, const kry_embed* pre);
}  // namespace kry

std::atomic<unsigned long long> g_kry_launches{0};

void kry_allow_max_smem(const void* func) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    KRY_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({func, dev})) return;
    int optin = 0;
    KRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes a;
    KRY_CUDA(cudaFuncGetAttributes(&a, func));
    KRY_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin - (int)a.sharedSizeBytes));
    done.insert({func, dev});
}

static void prof_clear(kry_ctx* ctx) {
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    ctx->prof_nvec.clear();
    ctx->prof_dbl.clear();
    for (int d = 0; d < 2; ++d) {
        ctx->prof_ms_acc[d] = 0.0;
        ctx->prof_calls_acc[d] = 0;
        ctx->prof_vec_acc[d] = 0;
    }
}

void DevBuf::ensure(size_t bytes) {
    if (bytes <= cap && p) return;
    release();
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        p = nullptr;
        cap = 0;
        (void)cudaGetLastError();
        throw KryError{KRY_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                       " bytes failed: " + cudaGetErrorString(e)};
    }
    cap = bytes;
}

void DevBuf::release() {
    if (p) cudaFreeAsync(p, stream);
    p = nullptr;
    cap = 0;
}

static void dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        throw KryError{KRY_ENOMEM, std::string("device allocation of ") + std::to_string(bytes) +
                                       " bytes failed: " + cudaGetErrorString(e)};
    }
}

namespace kry {
void ctx_trim(kry_ctx* ctx) {
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DevBuf* bufs[] = {&ctx->slab32, &ctx->slab64, &ctx->scal, &ctx->eig_c, &ctx->eig_z, &ctx->eig_d, &ctx->red, &ctx->tolbuf,
                      &ctx->kxbuf, &ctx->cbuf, &ctx->sbuf, &ctx->zbuf, &ctx->gbuf, &ctx->boot, &ctx->gk, &ctx->sites.grid32, &ctx->sites.grid64};
    for (DevBuf* b : bufs) b->release();
    for (auto& b : ctx->work) b.release();
    if (!ctx->sites.active) {
        // the whole-grid index lists are rebuilt on demand unless a site map needs them
        ctx->rowptr_full.release();
        ctx->colidx_full.release();
        ctx->full_n1 = ctx->full_n2 = 0;
    }
}
}  // namespace kry

// ------------------------------------------------------------------ mask compaction

// Observed cells per row (one block per row).
__global__ void k_row_counts(const uint8_t* __restrict__ mask, int n2, int* __restrict__ counts) {
    const int row = blockIdx.x;
    int c = 0;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) c += mask[(int64_t)row * n2 + j] != 0;
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        counts[row] = s;
    }
}

// Exclusive scan of the row counts into rowptr[0..n1] (one block, serial over warps).
__global__ void k_rowptr(const int* __restrict__ counts, int n1, int* __restrict__ rowptr) {
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < n1; ++i) {
            rowptr[i] = s;
            s += counts[i];
        }
        rowptr[n1] = s;
    }
}

// Observed cells of one row whose four neighbours are observed (beyond the
// grid edge counts as observed), added into *count (one block per row).
__global__ void k_interior_count(const uint8_t* __restrict__ mask, int n1, int n2,
                                 unsigned long long* __restrict__ count) {
    const int row = blockIdx.x;
    unsigned c = 0;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        const int64_t i = (int64_t)row * n2 + j;
        if (!mask[i]) continue;
        const bool up = row == 0 || mask[i - n2], down = row == n1 - 1 || mask[i + n2];
        const bool left = j == 0 || mask[i - 1], right = j == n2 - 1 || mask[i + 1];
        c += (up && down && left && right) ? 1u : 0u;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

// Ordered compaction of one row: colidx and cellidx of its observed cells.
__global__ void k_row_fill(const uint8_t* __restrict__ mask, int n2, const int* __restrict__ rowptr,
                           int* __restrict__ colidx, int* __restrict__ cellidx) {
    const int row = blockIdx.x;
    __shared__ int wsum[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = rowptr[row];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j0 = 0; j0 < n2; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool f = (j < n2) && mask[(int64_t)row * n2 + j] != 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[w] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int k = 0; k < w; ++k) off += wsum[k];
        const int pos = base + off + __popc(bal & ((1u << lane) - 1u));
        if (f) {
            colidx[pos] = j;
            cellidx[pos] = row * n2 + j;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < nw; ++k) t += wsum[k];
            base += t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ helpers

static kry_status fail(kry_ctx* ctx, kry_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return st;
}

template <class F>
static kry_status guarded(kry_ctx* ctx, F&& f) {
    if (!ctx) return KRY_EINVAL;
    try {
        KRY_CUDA(cudaSetDevice(ctx->device));
        ctx->err.clear();
        return f();
    } catch (const KryError& e) {
        ctx->err = e.msg;
        return e.st;
    } catch (const std::exception& e) {
        ctx->err = e.what();
        return KRY_ECUDA;
    }
}

static void check_cov(const kry_cov* cov) {
    KRY_REQUIRE(cov != nullptr, KRY_EINVAL, "cov is NULL");
    KRY_REQUIRE(cov->sigma2 >= 0 && isfinite(cov->sigma2), KRY_EINVAL, "sigma2 must be finite and >= 0");
    KRY_REQUIRE(cov->tau2 >= 0 && isfinite(cov->tau2), KRY_EINVAL, "tau2 must be finite and >= 0");
    KRY_REQUIRE(cov->range > 0 && isfinite(cov->range), KRY_EINVAL, "range must be finite and > 0");
    KRY_REQUIRE(cov->nu > 0 && cov->nu <= 8.0, KRY_EINVAL, "nu must be in (0, 8]");
    KRY_REQUIRE(cov->aniso_ratio > 0 && isfinite(cov->aniso_ratio), KRY_EINVAL, "aniso_ratio must be > 0");
    KRY_REQUIRE(isfinite(cov->aniso_angle), KRY_EINVAL, "aniso_angle must be finite");
}

static int pow2_at_least(int64_t x) {
    int M = 1;
    while (M < x) M *= 2;
    return M;
}

static void require_mask(kry_ctx* ctx) {
    KRY_REQUIRE(ctx->p > 0, KRY_EINVAL, "no observation mask set (kry_set_mask)");
}

static void check_embed(kry_ctx* ctx, const kry_embed* e) {
    KRY_REQUIRE(e != nullptr, KRY_EINVAL, "embedding is NULL");
    KRY_REQUIRE(e->ctx == ctx, KRY_EINVAL, "embedding belongs to another context");
    KRY_REQUIRE(e->n1 == ctx->n1 && e->n2 == ctx->n2, KRY_EINVAL, "embedding grid differs from the mask grid");
    require_mask(ctx);
}

// True if FP32 matvecs on this embedding run the length-specialised passes
// (their column pass reads the permuted eigenvalue copy lam32P).
static bool spec_column_pass(const kry_ctx* ctx, const kry_embed* e) {
    return ctx->use_spec && e->M1 >= 64 && e->M2 >= 64 && e->M1 <= 8192 && e->M2 <= 8192;
}

// True if FP32 iterates resolve the covariance whose embedding eigenvalues span
// [lam_lo, lam_hi] with nugget tau2 (KRY_F32_KAPPA_MAX).
static bool f32_resolves(double lam_lo, double lam_hi, double tau2) {
    const double lmax = std::max(fabs(lam_lo), fabs(lam_hi));
    return tau2 > 0.0 && (lmax + tau2) / tau2 <= KRY_F32_KAPPA_MAX;
}

// promote (prec = KRY_AUTO in kry_opts): an FP32 request whose conditioning
// FP32 cannot resolve gets an FP64 embedding (and counts in ctx->promoted).
static kry_embed* make_embed(kry_ctx* ctx, const kry_cov* cov, kry_prec prec, bool promote = false) {
    check_cov(cov);
    require_mask(ctx);
    KRY_REQUIRE(prec == KRY_F32 || prec == KRY_F64, KRY_EINVAL, "prec must be KRY_F32 or KRY_F64");
    kry_embed* e = new kry_embed();
    e->ctx = ctx;
    e->device = ctx->device;
    e->n1 = ctx->n1;
    e->n2 = ctx->n2;
    e->M1 = pow2_at_least(2 * (int64_t)ctx->n1);
    e->M2 = pow2_at_least(2 * (int64_t)ctx->n2);
    e->cov = *cov;
    e->prec = prec;
    e->stream = ctx->stream;
    try {
        kry::compute_eigs(ctx, *cov, ctx->n1, ctx->n2, ctx->dx1, ctx->dx2, e->M1, e->M2, &e->lam_min, &e->lam_max);
        if (promote && prec == KRY_F32 && !f32_resolves(e->lam_min, e->lam_max, cov->tau2)) {
            prec = KRY_F64;
            e->prec = KRY_F64;
            ++ctx->promoted;
        }
        const size_t MM = (size_t)e->M1 * e->M2;
        dev_alloc((void**)&e->lam64T, MM * sizeof(double), ctx->stream);
        if (prec == KRY_F32) dev_alloc((void**)&e->lam32T, MM * sizeof(float), ctx->stream);
        if (prec == KRY_F32 && spec_column_pass(ctx, e)) dev_alloc((void**)&e->lam32P, MM * sizeof(float), ctx->stream);
        kry::store_embedding(ctx, e, 0);
    } catch (...) {
        if (e->lam64T) cudaFreeAsync(e->lam64T, ctx->stream);
        if (e->lam32T) cudaFreeAsync(e->lam32T, ctx->stream);
        if (e->lam32P) cudaFreeAsync(e->lam32P, ctx->stream);
        delete e;
        throw;
    }
    return e;
}

// The precision a kry_opts call starts from (KRY_AUTO starts from FP32), and
// its embedding: KRY_AUTO promotes a setting FP32 does not resolve to FP64.
static kry_prec base_prec(const kry_opts* o) { return o->prec == KRY_AUTO ? KRY_F32 : o->prec; }
static kry_embed* make_embed_opts(kry_ctx* ctx, const kry_cov* cov, const kry_opts* o) {
    return make_embed(ctx, cov, base_prec(o), o->prec == KRY_AUTO);
}

// CG preconditioner for one covariance setting (kry_opts.precond) of a solve
// in precision prec: an FP32
// embedding whose matvec applies M^-1 = A (S + tau2 I)^-1 A^T, S the circulant
// embedding of sigma2 Sigma on the torus: eigenvalues 1 / (max(Lambda, 0) +
// tau2), no nugget.  NULL when it does not apply: FP64 solves, several
// settings, tau2 = 0, and irregular sites (with Wendland weights, close sites
// give nearly equal rows of A, so A (S + tau2 I)^-1 A^T is nearly singular and
// preconditioned CG stalls: measured, 12,000 sites on a 128^2 grid).
static kry_embed* make_precond_embed(kry_ctx* ctx, const kry_cov* cov, const kry_opts* o, kry_prec prec,
                                     int ntheta) {
    if (!o->precond || prec != KRY_F32 || ntheta != 1 || !(cov->tau2 > 0.0) || ctx->sites.active) return nullptr;
    // automatic choice: clustered gaps (measured on 512^2 masks: at an interior
    // share of 0.4 and more the preconditioned solve was the faster one)
    if (o->precond == 2 && ctx->interior < KRY_PRECOND_AUTO_INTERIOR) return nullptr;
    kry_embed* e = new kry_embed();
    e->ctx = ctx;
    e->device = ctx->device;
    e->n1 = ctx->n1;
    e->n2 = ctx->n2;
    e->M1 = pow2_at_least(2 * (int64_t)ctx->n1);
    e->M2 = pow2_at_least(2 * (int64_t)ctx->n2);
    e->cov = *cov;
    e->cov.tau2 = 0.0;
    e->prec = KRY_F32;
    e->stream = ctx->stream;
    try {
        kry::compute_eigs(ctx, *cov, ctx->n1, ctx->n2, ctx->dx1, ctx->dx2, e->M1, e->M2, &e->lam_min, &e->lam_max);
        kry::invert_eigs(ctx, e->M1, e->M2, cov->tau2);
        const size_t MM = (size_t)e->M1 * e->M2;
        dev_alloc((void**)&e->lam64T, MM * sizeof(double), ctx->stream);
        dev_alloc((void**)&e->lam32T, MM * sizeof(float), ctx->stream);
        if (spec_column_pass(ctx, e)) dev_alloc((void**)&e->lam32P, MM * sizeof(float), ctx->stream);
        kry::store_embedding(ctx, e, 0);
    } catch (...) {
        if (e->lam64T) cudaFreeAsync(e->lam64T, ctx->stream);
        if (e->lam32T) cudaFreeAsync(e->lam32T, ctx->stream);
        if (e->lam32P) cudaFreeAsync(e->lam32P, ctx->stream);
        delete e;
        throw;
    }
    return e;
}

namespace kry {
kry_embed* make_embed_internal(kry_ctx* ctx, const kry_cov* cov, kry_prec prec) { return make_embed(ctx, cov, prec); }
}  // namespace kry

// Stream-ordered release on stream s (the creating context's stream while it
// lives; the legacy stream from kry_embed_free, whose context may be gone).
static void free_embed(kry_embed* e, cudaStream_t s) {
    if (!e) return;
    if (e->lam64T) cudaFreeAsync(e->lam64T, s);
    if (e->lam32T) cudaFreeAsync(e->lam32T, s);
    if (e->lam32P) cudaFreeAsync(e->lam32P, s);
    if (e->tau2_dev) cudaFreeAsync(e->tau2_dev, s);
    delete e;
}
static void free_embed(kry_embed* e) {
    if (e) free_embed(e, e->stream);
}

namespace kry {
void free_embed_internal(kry_embed* e) { free_embed(e); }
}  // namespace kry

// Several covariance settings on the grid of the mask in one embedding:
// eigenvalue blocks back to back, per-setting nuggets on the device.
static kry_embed* make_embed_batch(kry_ctx* ctx, const kry_cov* thetas, int ntheta, kry_prec prec) {
    require_mask(ctx);
    for (int t = 0; t < ntheta; ++t) check_cov(&thetas[t]);
    kry_embed* e = new kry_embed();
    e->ctx = ctx;
    e->device = ctx->device;
    e->n1 = ctx->n1;
    e->n2 = ctx->n2;
    e->M1 = pow2_at_least(2 * (int64_t)ctx->n1);
    e->M2 = pow2_at_least(2 * (int64_t)ctx->n2);
    e->cov = thetas[0];
    e->prec = prec;
    e->stream = ctx->stream;
    e->ntheta = ntheta;
    const size_t MM = (size_t)e->M1 * e->M2;
    e->lam_stride = (int64_t)MM;
    try {
        dev_alloc((void**)&e->lam64T, ntheta * MM * sizeof(double), ctx->stream);
        if (prec == KRY_F32) dev_alloc((void**)&e->lam32T, ntheta * MM * sizeof(float), ctx->stream);
        if (prec == KRY_F32 && spec_column_pass(ctx, e))
            dev_alloc((void**)&e->lam32P, ntheta * MM * sizeof(float), ctx->stream);
        dev_alloc((void**)&e->tau2_dev, ntheta * sizeof(double), ctx->stream);
        std::vector<double> t2(ntheta);
        for (int t = 0; t < ntheta; ++t) {
            double lo, hi;
            kry::compute_eigs(ctx, thetas[t], ctx->n1, ctx->n2, ctx->dx1, ctx->dx2, e->M1, e->M2, &lo, &hi);
            kry::store_embedding(ctx, e, t);
            t2[t] = thetas[t].tau2;
            if (t == 0 || lo / hi < e->lam_min / e->lam_max) {
                e->lam_min = lo;
                e->lam_max = hi;
            }
        }
        KRY_CUDA(cudaMemcpyAsync(e->tau2_dev, t2.data(), ntheta * sizeof(double), cudaMemcpyHostToDevice,
                                 ctx->stream));
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
        free_embed(e);
        throw;
    }
    return e;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

kry_status kry_create(kry_ctx** out, int device, void* cuda_stream) {
    if (!out) return KRY_EINVAL;
    *out = nullptr;
    kry_ctx* ctx = new kry_ctx();
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    kry_status st = guarded(ctx, [&]() -> kry_status {
        int ndev = 0;
        KRY_CUDA(cudaGetDeviceCount(&ndev));
        KRY_REQUIRE(device >= 0 && device < ndev, KRY_EINVAL, "no such CUDA device");
        KRY_CUDA(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
        KRY_CUDA(cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
        // every scratch buffer is stream-ordered on the context stream; keep freed
        // pool memory cached in this process instead of returning it at each sync
        DevBuf* bufs[] = {&ctx->rowptr, &ctx->colidx, &ctx->cellidx, &ctx->tw32, &ctx->tw64, &ctx->twt32, &ctx->slab32,
                          &ctx->slab64, &ctx->scal, &ctx->eig_c, &ctx->eig_z, &ctx->eig_d, &ctx->red, &ctx->tolbuf,
                          &ctx->kxbuf, &ctx->cbuf, &ctx->sbuf, &ctx->zbuf, &ctx->gbuf, &ctx->boot, &ctx->gk, &ctx->rowptr_full, &ctx->colidx_full,
                      &ctx->sites.corner, &ctx->sites.w64, &ctx->sites.w32, &ctx->sites.cellptr, &ctx->sites.ent_site,
                      &ctx->sites.ent_w64, &ctx->sites.ent_w32, &ctx->sites.cnt, &ctx->sites.grid32, &ctx->sites.grid64};
        for (DevBuf* b : bufs) b->stream = ctx->stream;
        for (auto& b : ctx->work) b.stream = ctx->stream;
        cudaMemPool_t pool;
        KRY_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
        uint64_t keep = UINT64_MAX;
        KRY_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        KRY_CUDA(cudaMallocHost(&ctx->host_pinned, 4096 * sizeof(double)));
        kry::init_twiddles(ctx);
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        return KRY_OK;
    });
    if (st != KRY_OK) {
        fprintf(stderr, "kry_create: %s\n", ctx->err.c_str());
        kry_destroy(ctx);
        return st;
    }
    *out = ctx;
    return KRY_OK;
}

void kry_destroy(kry_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    DevBuf* bufs[] = {&ctx->rowptr, &ctx->colidx, &ctx->cellidx, &ctx->tw32, &ctx->tw64, &ctx->twt32, &ctx->slab32,
                      &ctx->slab64, &ctx->scal, &ctx->eig_c, &ctx->eig_z, &ctx->eig_d, &ctx->red, &ctx->tolbuf,
                      &ctx->kxbuf, &ctx->cbuf, &ctx->sbuf, &ctx->zbuf, &ctx->gbuf, &ctx->boot, &ctx->gk, &ctx->rowptr_full, &ctx->colidx_full,
                      &ctx->sites.corner, &ctx->sites.w64, &ctx->sites.w32, &ctx->sites.cellptr, &ctx->sites.ent_site,
                      &ctx->sites.ent_w64, &ctx->sites.ent_w32, &ctx->sites.cnt, &ctx->sites.grid32, &ctx->sites.grid64};
    for (DevBuf* b : bufs) b->release();
    for (auto& b : ctx->work) b.release();
    prof_clear(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    delete ctx;
}

const char* kry_last_error(const kry_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

kry_status kry_set_mask(kry_ctx* ctx, const kry_grid* grid, const uint8_t* mask_dev, int64_t* p_out) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(grid && mask_dev, KRY_EINVAL, "grid and mask_dev must not be NULL");
        KRY_REQUIRE(grid->n1 >= 4 && grid->n2 >= 4, KRY_EUNSUPPORTED, "grid sides must be >= 4");
        KRY_REQUIRE(grid->n1 <= KRY_MAX_N && grid->n2 <= KRY_MAX_N, KRY_EUNSUPPORTED, "grid sides must be <= 4096");
        KRY_REQUIRE(grid->dx1 > 0 && grid->dx2 > 0, KRY_EINVAL, "cell sizes must be > 0");
        const int n1 = grid->n1, n2 = grid->n2;
        ctx->p = 0;
        ctx->sites.active = false;
        ctx->rowptr.ensure((size_t)(n1 + 1) * sizeof(int));
        ctx->colidx.ensure((size_t)n1 * n2 * sizeof(int));
        ctx->cellidx.ensure((size_t)n1 * n2 * sizeof(int));
        ctx->red.ensure((size_t)(n1 + 4) * sizeof(int) + sizeof(unsigned long long));
        int* counts = ctx->red.as<int>();
        k_row_counts<<<n1, 256, 0, ctx->stream>>>(mask_dev, n2, counts);
        KRY_CHECK_LAUNCH();
        k_rowptr<<<1, 32, 0, ctx->stream>>>(counts, n1, ctx->rowptr.as<int>());
        KRY_CHECK_LAUNCH();
        k_row_fill<<<n1, 256, 0, ctx->stream>>>(mask_dev, n2, ctx->rowptr.as<int>(), ctx->colidx.as<int>(),
                                                ctx->cellidx.as<int>());
        KRY_CHECK_LAUNCH();
        unsigned long long* icount = reinterpret_cast<unsigned long long*>(ctx->red.as<int>() + ((n1 + 2) & ~1));
        KRY_CUDA(cudaMemsetAsync(icount, 0, sizeof(unsigned long long), ctx->stream));
        k_interior_count<<<n1, 256, 0, ctx->stream>>>(mask_dev, n1, n2, icount);
        KRY_CHECK_LAUNCH();
        int* hp = reinterpret_cast<int*>(ctx->host_pinned);
        KRY_CUDA(cudaMemcpyAsync(hp, ctx->rowptr.as<int>() + n1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned + 1, icount, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                 ctx->stream));
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        const int64_t p = hp[0];
        const unsigned long long interior = *reinterpret_cast<unsigned long long*>(ctx->host_pinned + 1);
        KRY_REQUIRE(p >= 1, KRY_EINVAL, "mask has no observed cell");
        ctx->interior = (double)interior / (double)p;
        ctx->n1 = n1;
        ctx->n2 = n2;
        ctx->dx1 = grid->dx1;
        ctx->dx2 = grid->dx2;
        ctx->p = p;
        if (p_out) *p_out = p;
        return KRY_OK;
    });
}

kry_status kry_mask_interior(kry_ctx* ctx, double* interior) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(interior != nullptr, KRY_EINVAL, "interior must not be NULL");
        *interior = (ctx->p > 0 && !ctx->sites.active) ? ctx->interior : 0.0;
        return KRY_OK;
    });
}

kry_status kry_promoted(kry_ctx* ctx, int64_t* count) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(count != nullptr, KRY_EINVAL, "count must not be NULL");
        *count = ctx->promoted;
        return KRY_OK;
    });
}

kry_status kry_set_sites(kry_ctx* ctx, const kry_grid* grid, const double* sites_dev, int64_t nsite) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(grid && sites_dev, KRY_EINVAL, "grid and sites_dev must not be NULL");
        KRY_REQUIRE(grid->n1 >= 4 && grid->n2 >= 4, KRY_EUNSUPPORTED, "grid sides must be >= 4");
        KRY_REQUIRE(grid->n1 <= KRY_MAX_N && grid->n2 <= KRY_MAX_N, KRY_EUNSUPPORTED, "grid sides must be <= 4096");
        KRY_REQUIRE(grid->dx1 > 0 && grid->dx2 > 0, KRY_EINVAL, "cell sizes must be > 0");
        KRY_REQUIRE(nsite >= 1 && nsite <= ((int64_t)1 << 29), KRY_EINVAL, "nsite must be in [1, 2^29]");
        ctx->p = 0;
        ctx->sites.active = false;
        const bool ok = kry::build_sites(ctx, grid->n1, grid->n2, grid->dx1, grid->dx2, sites_dev, nsite);
        KRY_REQUIRE(ok, KRY_EINVAL, "a site lies outside the domain [0, n1 dx1] x [0, n2 dx2] or is not finite");
        ctx->n1 = grid->n1;
        ctx->n2 = grid->n2;
        ctx->dx1 = grid->dx1;
        ctx->dx2 = grid->dx2;
        ctx->p = nsite;
        ctx->sites.active = true;
        return KRY_OK;
    });
}

kry_status kry_embed_eigs(kry_ctx* ctx, const kry_cov* cov, kry_prec prec, kry_embed** out, double* min_over_max) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(out != nullptr, KRY_EINVAL, "out is NULL");
        *out = nullptr;
        kry_embed* e = make_embed(ctx, cov, prec);
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        if (min_over_max) *min_over_max = (e->lam_max != 0.0) ? e->lam_min / e->lam_max : 0.0;
        *out = e;
        return KRY_OK;
    });
}

void kry_embed_free(kry_embed* e) {
    if (!e) return;
    // the owning context (and its stream) may be gone: free in order on the
    // legacy stream after the device has finished the embedding's work
    cudaSetDevice(e->device);
    cudaDeviceSynchronize();
    free_embed(e, (cudaStream_t)0);
}

kry_status kry_matvec(kry_ctx* ctx, const kry_embed* e, const void* v_dev, void* out_dev, int32_t nvec, int64_t ld) {
    return guarded(ctx, [&]() -> kry_status {
        check_embed(ctx, e);
        KRY_REQUIRE(nvec >= 0 && ld >= ctx->p, KRY_EINVAL, "need nvec >= 0 and ld >= p");
        if (nvec == 0) return KRY_OK;
        KRY_REQUIRE(v_dev && out_dev, KRY_EINVAL, "v_dev and out_dev must not be NULL");
        if (e->prec == KRY_F64)
            kry::matvec_ex<double>(ctx, e, static_cast<const double*>(v_dev), ld, nullptr, static_cast<double*>(out_dev),
                                   ld, nvec, nullptr, 0);
        else
            kry::matvec_ex<float>(ctx, e, static_cast<const float*>(v_dev), ld, nullptr, static_cast<float*>(out_dev),
                                  ld, nvec, nullptr, 0);
        return KRY_OK;
    });
}

static void mean_se(const std::vector<double>& v, double* mean, double* se) {
    const int n = (int)v.size();
    double s = 0.0;
    for (double x : v) s += x;
    const double m = s / n;
    double q = 0.0;
    for (double x : v) q += (x - m) * (x - m);
    *mean = m;
    if (se) *se = (n > 1) ? sqrt(q / (n - 1) / n) : 0.0;
}

kry_status kry_logdet(kry_ctx* ctx, const kry_embed* e, int32_t nprobe, int32_t nsteps, uint64_t seed, int32_t reorth,
                      double* logdet, double* stderr_out, double* per_probe) {
    return guarded(ctx, [&]() -> kry_status {
        check_embed(ctx, e);
        KRY_REQUIRE(logdet != nullptr, KRY_EINVAL, "logdet is NULL");
        KRY_REQUIRE(nprobe >= 1 && nsteps >= 1, KRY_EINVAL, "need nprobe >= 1 and nsteps >= 1");
        KRY_REQUIRE(reorth == 0 || reorth == 1, KRY_EINVAL, "reorth must be 0 or 1");
        std::vector<double> vals(nprobe);
        kry::logdet(ctx, e, nprobe, nsteps, seed, reorth != 0, vals.data());
        double se = 0.0;
        mean_se(vals, logdet, &se);
        if (stderr_out) *stderr_out = se;
        if (per_probe) memcpy(per_probe, vals.data(), nprobe * sizeof(double));
        for (double v : vals)
            if (!isfinite(v)) return fail(ctx, KRY_ENAN, "log-det quadrature produced NaN/Inf");
        return KRY_OK;
    });
}

kry_status kry_solve(kry_ctx* ctx, const kry_embed* e, const double* B_dev, double* X_dev, int32_t nrhs, int64_t ld,
                     double rtol, int32_t maxit, int32_t* iters, double* relres) {
    return guarded(ctx, [&]() -> kry_status {
        check_embed(ctx, e);
        KRY_REQUIRE(B_dev && X_dev, KRY_EINVAL, "B_dev and X_dev must not be NULL");
        KRY_REQUIRE(nrhs >= 1 && nrhs <= 1024 && ld >= ctx->p, KRY_EINVAL, "need 1 <= nrhs <= 1024 and ld >= p");
        KRY_REQUIRE(rtol > 0 && maxit >= 1, KRY_EINVAL, "need rtol > 0 and maxit >= 1");
        kry::SolveInfo si = kry::solve(ctx, e, B_dev, ld, X_dev, ld, nrhs, rtol, maxit);
        if (iters) *iters = si.iters;
        if (relres) *relres = si.relres;
        if (!isfinite(si.relres)) return fail(ctx, KRY_ENAN, "CG residual is NaN/Inf");
        if (!si.converged) return fail(ctx, KRY_ENOCONV, "CG did not reach rtol");
        return KRY_OK;
    });
}

kry_status kry_solve_pre(kry_ctx* ctx, const kry_embed* e, const double* B_dev, double* X_dev, int32_t nrhs,
                         int64_t ld, double rtol, int32_t maxit, int32_t* iters, double* relres) {
    return guarded(ctx, [&]() -> kry_status {
        check_embed(ctx, e);
        KRY_REQUIRE(B_dev && X_dev, KRY_EINVAL, "B_dev and X_dev must not be NULL");
        KRY_REQUIRE(nrhs >= 1 && nrhs <= 1024 && ld >= ctx->p, KRY_EINVAL, "need 1 <= nrhs <= 1024 and ld >= p");
        KRY_REQUIRE(rtol > 0 && maxit >= 1, KRY_EINVAL, "need rtol > 0 and maxit >= 1");
        KRY_REQUIRE(e->ntheta == 1, KRY_EINVAL, "one covariance setting per embedding");
        kry_opts o{};
        o.prec = e->prec;
        o.precond = 1;
        kry_embed* pre = make_precond_embed(ctx, &e->cov, &o, e->prec, 1);
        kry::SolveInfo si;
        try {
            si = kry::solve(ctx, e, B_dev, ld, X_dev, ld, nrhs, rtol, maxit, 0, pre);
        } catch (...) {
            free_embed(pre);
            throw;
        }
        free_embed(pre);
        if (iters) *iters = si.iters;
        if (relres) *relres = si.relres;
        if (!isfinite(si.relres)) return fail(ctx, KRY_ENAN, "CG residual is NaN/Inf");
        if (!si.converged) return fail(ctx, KRY_ENOCONV, "CG did not reach rtol");
        return KRY_OK;
    });
}

static void check_opts(const kry_opts* o) {
    KRY_REQUIRE(o != nullptr && o->precond >= 0 && o->precond <= 2, KRY_EINVAL, "opts->precond must be 0, 1 or 2");
    KRY_REQUIRE(o != nullptr, KRY_EINVAL, "opts is NULL");
    KRY_REQUIRE(o->prec == KRY_F32 || o->prec == KRY_F64 || o->prec == KRY_AUTO, KRY_EINVAL, "opts->prec invalid");
    KRY_REQUIRE(o->nprobe >= 1 && o->nsteps >= 1, KRY_EINVAL, "need nprobe >= 1 and nsteps >= 1");
    KRY_REQUIRE(o->rtol > 0 && o->maxit >= 1, KRY_EINVAL, "need rtol > 0 and maxit >= 1");
    KRY_REQUIRE(o->reorth == 0 || o->reorth == 1, KRY_EINVAL, "opts->reorth must be 0 or 1");
}

// [y, X] packed into one (p x (ncov+1)) FP64 block and its solve Z = K^-1 [y, X]
// (preconditioned when o->precond asks for it and it applies).
static kry::SolveInfo solve_yx(kry_ctx* ctx, const kry_embed* e, const double* y, const double* X, int ncov,
                               const kry_opts* o, double** V_out, double** Z_out) {
    const int64_t p = ctx->p;
    const int nc = ncov + 1;
    ctx->zbuf.ensure((size_t)2 * nc * p * sizeof(double));
    double* V = ctx->zbuf.as<double>();
    double* Z = V + (size_t)nc * p;
    KRY_CUDA(cudaMemcpyAsync(V, y, p * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    KRY_CUDA(cudaMemcpyAsync(V + p, X, (size_t)ncov * p * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    *V_out = V;
    *Z_out = Z;
    kry_embed* pre = make_precond_embed(ctx, &e->cov, o, e->prec, 1);
    kry::SolveInfo si;
    try {
        si = kry::solve(ctx, e, V, p, Z, p, nc, o->rtol, o->maxit, 0, pre);
    } catch (...) {
        free_embed(pre);
        throw;
    }
    free_embed(pre);
    return si;
}

kry_status kry_profile_loglik(kry_ctx* ctx, const double* y_dev, const double* X_dev, int32_t ncov,
                              const kry_cov* thetas, int32_t ntheta, const kry_opts* opts, double* loglik,
                              double* beta, double* logdet, double* logdet_se) {
    return guarded(ctx, [&]() -> kry_status {
        require_mask(ctx);
        check_opts(opts);
        KRY_REQUIRE(y_dev && X_dev && thetas && loglik, KRY_EINVAL, "y_dev, X_dev, thetas, loglik must not be NULL");
        KRY_REQUIRE(ncov >= 1 && ncov <= KRY_MAX_COV, KRY_EINVAL, "ncov must be in [1, 8]");
        KRY_REQUIRE(ntheta >= 1, KRY_EINVAL, "ntheta must be >= 1");
        for (int t = 0; t < ntheta; ++t) check_cov(&thetas[t]);
        const int64_t p = ctx->p;
        const int nc = ncov + 1;
        const int ncp = nc + (nc & 1);   // right-hand sides per setting, padded to pair up
        const bool batched = ntheta > 1 && opts->nprobe % 2 == 0;
        // settings per group: keep the batched vectors within ~2048 (log-det) per launch sequence
        const int group = batched ? std::max(1, std::min<int>(ntheta, 2048 / opts->nprobe)) : 1;
        // an FP32 batch holds only settings that FP32 resolves (KRY_F32_KAPPA_MAX);
        // the others run alone, promoted to FP64
        std::vector<std::vector<int>> groups;
        {
            std::vector<int> in_batch, alone;
            for (int t = 0; t < ntheta; ++t) {
                bool ok = true;
                if (batched && opts->prec == KRY_AUTO) {
                    double lo, hi;
                    kry::compute_eigs(ctx, thetas[t], ctx->n1, ctx->n2, ctx->dx1, ctx->dx2,
                                      pow2_at_least(2 * (int64_t)ctx->n1), pow2_at_least(2 * (int64_t)ctx->n2), &lo,
                                      &hi);
                    ok = f32_resolves(lo, hi, thetas[t].tau2);
                }
                (ok ? in_batch : alone).push_back(t);
            }
            for (size_t i = 0; i < in_batch.size(); i += group)
                groups.emplace_back(in_batch.begin() + i, in_batch.begin() + std::min(in_batch.size(), i + group));
            for (int t : alone) groups.push_back({t});
        }
        kry_status worst = KRY_OK;
        for (const std::vector<int>& gi : groups) {
            const int ng = (int)gi.size();
            std::vector<kry_cov> th(ng);
            for (int t = 0; t < ng; ++t) th[t] = thetas[gi[t]];
            kry_embed* e = (ng > 1) ? make_embed_batch(ctx, th.data(), ng, base_prec(opts))
                                    : make_embed_opts(ctx, &th[0], opts);
            try {
                // log-determinants: ng settings x nprobe probes in one batched Lanczos
                std::vector<double> vals((size_t)ng * opts->nprobe);
                if (ng > 1)
                    kry::logdet_batched(ctx, e, opts->nprobe, opts->nsteps, opts->seed, opts->reorth != 0, vals.data());
                else
                    kry::logdet(ctx, e, opts->nprobe, opts->nsteps, opts->seed, opts->reorth != 0, vals.data());
                // right-hand sides [y, X] (zero-padded to ncp columns) repeated for each setting
                ctx->zbuf.ensure((size_t)(nc + 2 * (size_t)ng * ncp) * p * sizeof(double));
                double* V = ctx->zbuf.as<double>();
                double* Vrep = V + (size_t)nc * p;
                double* Z = Vrep + (size_t)ng * ncp * p;
                KRY_CUDA(cudaMemcpyAsync(V, y_dev, p * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
                KRY_CUDA(cudaMemcpyAsync(V + p, X_dev, (size_t)ncov * p * sizeof(double), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
                for (int t = 0; t < ng; ++t) {
                    double* blk = Vrep + (size_t)t * ncp * p;
                    KRY_CUDA(cudaMemcpyAsync(blk, V, (size_t)nc * p * sizeof(double), cudaMemcpyDeviceToDevice,
                                             ctx->stream));
                    if (ncp > nc)
                        KRY_CUDA(cudaMemsetAsync(blk + (size_t)nc * p, 0, p * sizeof(double), ctx->stream));
                }
                kry_embed* pre = make_precond_embed(ctx, &th[0], opts, e->prec, ng);
                kry::SolveInfo si;
                try {
                    si = kry::solve(ctx, e, Vrep, p, Z, p, ng * ncp, opts->rtol, opts->maxit, ng > 1 ? ncp : 0, pre);
                } catch (...) {
                    free_embed(pre);
                    throw;
                }
                free_embed(pre);
                for (int t = 0; t < ng; ++t) {
                    std::vector<double> pv(vals.begin() + (size_t)t * opts->nprobe,
                                           vals.begin() + (size_t)(t + 1) * opts->nprobe);
                    double ld = 0, se = 0;
                    mean_se(pv, &ld, &se);
                    kry::GlsResult g = kry::gls(ctx, V, Z + (size_t)t * ncp * p, ncov, ld);
                    const int ti = gi[t];
                    loglik[ti] = g.loglik;
                    if (beta)
                        for (int c = 0; c < ncov; ++c) beta[(size_t)ti * ncov + c] = g.beta[c];
                    if (logdet) logdet[ti] = ld;
                    if (logdet_se) logdet_se[ti] = se;
                    if (!isfinite(g.loglik) || !g.ok) worst = KRY_ENAN;
                }
                if (!si.converged && worst == KRY_OK) worst = KRY_ENOCONV;
            } catch (...) {
                free_embed(e);
                throw;
            }
            free_embed(e);
        }
        if (worst == KRY_ENAN) return fail(ctx, worst, "log-likelihood is NaN/Inf or X^T K^-1 X is singular");
        if (worst == KRY_ENOCONV) return fail(ctx, worst, "CG did not reach rtol for some theta");
        return KRY_OK;
    });
}

}  // extern "C"

// Kriging means (and optional variances) from an embedding, the solve
// Z = K^-1 [y, X] and its GLS beta; shared by kry_krige and kry_loglik_krige.
static kry_status krige_from_solution(kry_ctx* ctx, kry_embed* e, const kry_cov& cov, const kry_opts* opts,
                                      const double* Z, int ncov, const kry::GlsResult& g, const kry::SolveInfo& si,
                                      const int64_t* cells_dev, const double* Xc_dev, int64_t ncell,
                                      const double* sites_dev, const double* Xs_dev, int64_t nsite,
                                      double* mean_cells_dev, double* mean_sites_dev, double* var_cells_dev) {
    const int64_t p = ctx->p;
    const int64_t N = (int64_t)ctx->n1 * ctx->n2;
    ctx->gbuf.ensure((size_t)(N + p + KRY_MAX_COV + 1) * sizeof(double));
    double* grid = ctx->gbuf.as<double>();
    double* w = grid + N;
    double* bdev = w + p;
    int* bad = reinterpret_cast<int*>(bdev + KRY_MAX_COV);
    KRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    KRY_CUDA(cudaMemcpyAsync(bdev, g.beta, ncov * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    kry::resid_weights(ctx, Z, ncov, bdev, w);
    if (ncell > 0) {
        // sigma2 Sigma A^T w on every grid cell (FP64 FFT path, no nugget)
        kry::sigma_to_grid64(ctx, e, w, grid, 1, p);
        kry::krige_launch_cells(ctx, grid, cells_dev, ncell, Xc_dev, ncov, bdev, mean_cells_dev, bad);
    }
    kry::krige_launch_sites(ctx, cov, sites_dev, nsite, Xs_dev, ncov, bdev, w, mean_sites_dev);
    bool vok = true;
    if (var_cells_dev && ncell > 0) {
        // the targets' cross-covariance solves, preconditioned like [y, X] when opts asks for it
        kry_embed* pre = make_precond_embed(ctx, &cov, opts, e->prec, 1);
        try {
            vok = kry::krige_variances(ctx, e, cells_dev, ncell, var_cells_dev, opts->rtol, opts->maxit, pre);
        } catch (...) {
            free_embed(pre);
            throw;
        }
        free_embed(pre);
    }
    int* hbad = reinterpret_cast<int*>(ctx->host_pinned);
    KRY_CUDA(cudaMemcpyAsync(hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
    if (*hbad) return fail(ctx, KRY_EINVAL, "a target cell index lies outside the grid (its mean is NaN)");
    if (!g.ok) return fail(ctx, KRY_ENAN, "X^T K^-1 X is singular");
    if (!si.converged || !vok) return fail(ctx, KRY_ENOCONV, "CG did not reach rtol");
    return KRY_OK;
}

static void check_krige_args(const kry_ctx* ctx, const double* y_dev, const double* X_dev, int32_t ncov,
                             const int64_t* cells_dev, const double* Xc_dev, int64_t ncell, const double* sites_dev,
                             const double* Xs_dev, int64_t nsite, double* mean_cells_dev, double* mean_sites_dev,
                             double* var_cells_dev) {
    KRY_REQUIRE(!ctx->sites.active || (nsite == 0 && var_cells_dev == nullptr), KRY_EUNSUPPORTED,
                "with irregular sites (kry_set_sites) kriging covers grid cells only, without variances");
    KRY_REQUIRE(y_dev && X_dev, KRY_EINVAL, "y_dev and X_dev must not be NULL");
    KRY_REQUIRE(ncov >= 1 && ncov <= KRY_MAX_COV, KRY_EINVAL, "ncov must be in [1, 8]");
    KRY_REQUIRE(ncell >= 0 && nsite >= 0, KRY_EINVAL, "ncell and nsite must be >= 0");
    KRY_REQUIRE(ncell == 0 || (cells_dev && Xc_dev && mean_cells_dev), KRY_EINVAL,
                "cells_dev, Xc_dev and mean_cells_dev are required when ncell > 0");
    KRY_REQUIRE(nsite == 0 || (sites_dev && Xs_dev && mean_sites_dev), KRY_EINVAL,
                "sites_dev, Xs_dev and mean_sites_dev are required when nsite > 0");
}

extern "C" {

kry_status kry_krige(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts, const double* y_dev, const double* X_dev,
                     int32_t ncov, const int64_t* cells_dev, const double* Xc_dev, int64_t ncell,
                     const double* sites_dev, const double* Xs_dev, int64_t nsite, double* mean_cells_dev,
                     double* mean_sites_dev, double* var_cells_dev, double* beta_out) {
    return guarded(ctx, [&]() -> kry_status {
        require_mask(ctx);
        check_opts(opts);
        check_cov(cov);
        check_krige_args(ctx, y_dev, X_dev, ncov, cells_dev, Xc_dev, ncell, sites_dev, Xs_dev, nsite,
                         mean_cells_dev, mean_sites_dev, var_cells_dev);
        kry_embed* e = make_embed_opts(ctx, cov, opts);
        kry_status st = KRY_OK;
        try {
            double *V, *Z;
            kry::SolveInfo si = solve_yx(ctx, e, y_dev, X_dev, ncov, opts, &V, &Z);
            kry::GlsResult g = kry::gls(ctx, V, Z, ncov, 0.0);
            if (beta_out)
                for (int c = 0; c < ncov; ++c) beta_out[c] = g.beta[c];
            st = krige_from_solution(ctx, e, *cov, opts, Z, ncov, g, si, cells_dev, Xc_dev, ncell, sites_dev,
                                     Xs_dev, nsite, mean_cells_dev, mean_sites_dev, var_cells_dev);
        } catch (...) {
            free_embed(e);
            throw;
        }
        free_embed(e);
        return st;
    });
}

kry_status kry_loglik_krige(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts, const double* y_dev,
                            const double* X_dev, int32_t ncov, const int64_t* cells_dev, const double* Xc_dev,
                            int64_t ncell, const double* sites_dev, const double* Xs_dev, int64_t nsite,
                            double* mean_cells_dev, double* mean_sites_dev, double* var_cells_dev, double* loglik,
                            double* beta, double* logdet, double* logdet_se) {
    return guarded(ctx, [&]() -> kry_status {
        require_mask(ctx);
        check_opts(opts);
        check_cov(cov);
        KRY_REQUIRE(loglik != nullptr, KRY_EINVAL, "loglik must not be NULL");
        check_krige_args(ctx, y_dev, X_dev, ncov, cells_dev, Xc_dev, ncell, sites_dev, Xs_dev, nsite,
                         mean_cells_dev, mean_sites_dev, var_cells_dev);
        kry_embed* e = make_embed_opts(ctx, cov, opts);
        kry_status st = KRY_OK;
        try {
            std::vector<double> vals(opts->nprobe);
            kry::logdet(ctx, e, opts->nprobe, opts->nsteps, opts->seed, opts->reorth != 0, vals.data());
            double ld = 0, se = 0;
            mean_se(vals, &ld, &se);
            double *V, *Z;
            kry::SolveInfo si = solve_yx(ctx, e, y_dev, X_dev, ncov, opts, &V, &Z);
            kry::GlsResult g = kry::gls(ctx, V, Z, ncov, ld);
            *loglik = g.loglik;
            if (beta)
                for (int c = 0; c < ncov; ++c) beta[c] = g.beta[c];
            if (logdet) *logdet = ld;
            if (logdet_se) *logdet_se = se;
            st = krige_from_solution(ctx, e, *cov, opts, Z, ncov, g, si, cells_dev, Xc_dev, ncell, sites_dev,
                                     Xs_dev, nsite, mean_cells_dev, mean_sites_dev, var_cells_dev);
            if (st == KRY_OK && !isfinite(g.loglik)) st = fail(ctx, KRY_ENAN, "log-likelihood is NaN/Inf");
        } catch (...) {
            free_embed(e);
            throw;
        }
        free_embed(e);
        return st;
    });
}

kry_status kry_profile_enable(kry_ctx* ctx, int on) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        prof_clear(ctx);
        ctx->prof_on = on != 0;
        return KRY_OK;
    });
}

kry_status kry_profile_read(kry_ctx* ctx, int32_t prec, int64_t* calls, int64_t* vectors, double* total_ms) {
    return guarded(ctx, [&]() -> kry_status {
        KRY_REQUIRE(calls && vectors && total_ms, KRY_EINVAL, "output pointers must not be NULL");
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        int64_t c = 0, v = 0;
        double ms = 0.0;
        for (size_t i = 0; i < ctx->prof_nvec.size(); ++i) {
            if (ctx->prof_dbl[i] != (prec == KRY_F64 ? 1 : 0)) continue;
            float t = 0.f;
            KRY_CUDA(cudaEventElapsedTime(&t, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
            ms += t;
            ++c;
            v += ctx->prof_nvec[i];
        }
        const int d = prec == KRY_F64 ? 1 : 0;
        *calls = c + ctx->prof_calls_acc[d];
        *vectors = v + ctx->prof_vec_acc[d];
        *total_ms = ms + ctx->prof_ms_acc[d];
        return KRY_OK;
    });
}

uint64_t kry_launch_count(void) { return g_kry_launches.load(); }

kry_status kry_sample_size(kry_ctx* ctx, const kry_cov* cov, int32_t* M1, int32_t* M2) {
    return guarded(ctx, [&]() -> kry_status {
        check_cov(cov);
        require_mask(ctx);
        KRY_REQUIRE(M1 && M2, KRY_EINVAL, "M1 and M2 must not be NULL");
        int m1 = pow2_at_least(2 * (int64_t)ctx->n1), m2 = pow2_at_least(2 * (int64_t)ctx->n2);
        for (int d = 0; d <= 3; ++d) {
            if (m1 > KRY_MAX_M || m2 > KRY_MAX_M) break;
            double lo, hi;
            kry::compute_eigs(ctx, *cov, ctx->n1, ctx->n2, ctx->dx1, ctx->dx2, m1, m2, &lo, &hi);
            *M1 = m1;
            *M2 = m2;
            if (lo >= -1e-10 * hi) return KRY_OK;
            m1 *= 2;
            m2 *= 2;
        }
        return fail(ctx, KRY_ENOTPSD, "no embedding up to the size limit is positive semi-definite");
    });
}

kry_status kry_sample(kry_ctx* ctx, const kry_cov* cov, int32_t M1, int32_t M2, const double* xi_dev,
                      double* out_dev) {
    return guarded(ctx, [&]() -> kry_status {
        check_cov(cov);
        require_mask(ctx);
        KRY_REQUIRE(xi_dev && out_dev, KRY_EINVAL, "xi_dev and out_dev must not be NULL");
        KRY_REQUIRE(M1 >= 2 * ctx->n1 && M2 >= 2 * ctx->n2 && M1 <= KRY_MAX_M && M2 <= KRY_MAX_M &&
                        (M1 & (M1 - 1)) == 0 && (M2 & (M2 - 1)) == 0,
                    KRY_EINVAL, "M1, M2 must be powers of two with 2 n_d <= M_d <= 8192");
        kry::sample_field(ctx, *cov, M1, M2, xi_dev, out_dev);
        return KRY_OK;
    });
}

kry_status kry_bootstrap_var(kry_ctx* ctx, const kry_cov* cov, const kry_opts* opts, int32_t nrep, int32_t M1,
                             int32_t M2, const double* xi_dev, const double* eps_dev, const int64_t* cells_dev,
                             int64_t ncell, double* var_dev) {
    return guarded(ctx, [&]() -> kry_status {
        check_cov(cov);
        check_opts(opts);
        require_mask(ctx);
        KRY_REQUIRE(!ctx->sites.active, KRY_EUNSUPPORTED, "the bootstrap needs an observation mask (kry_set_mask)");
        KRY_REQUIRE(nrep >= 1, KRY_EINVAL, "nrep must be >= 1");
        KRY_REQUIRE(xi_dev && eps_dev, KRY_EINVAL, "xi_dev and eps_dev must not be NULL");
        KRY_REQUIRE(ncell >= 0 && (ncell == 0 || (cells_dev && var_dev)), KRY_EINVAL,
                    "cells_dev and var_dev are required when ncell > 0");
        KRY_REQUIRE(M1 >= 2 * ctx->n1 && M2 >= 2 * ctx->n2 && M1 <= KRY_MAX_M && M2 <= KRY_MAX_M &&
                        (M1 & (M1 - 1)) == 0 && (M2 & (M2 - 1)) == 0,
                    KRY_EINVAL, "M1, M2 must be powers of two with 2 n_d <= M_d <= 8192");
        const int64_t N = (int64_t)ctx->n1 * ctx->n2, p = ctx->p;
        ctx->boot.ensure(((size_t)2 * nrep * N + (size_t)2 * nrep * p) * sizeof(double) + 16);
        double* G = ctx->boot.as<double>();       // sampled fields x_b on the grid
        double* H = G + (size_t)nrep * N;         // predictions sigma^2 Sigma A^T K^-1 r_b on the grid
        double* R = H + (size_t)nrep * N;         // r_b = A x_b + tau eps_b
        double* Wd = R + (size_t)nrep * p;        // K^-1 r_b
        int* bad = reinterpret_cast<int*>(Wd + (size_t)nrep * p);
        KRY_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
        for (int b = 0; b < nrep; ++b)
            kry::sample_field(ctx, *cov, M1, M2, xi_dev + (size_t)b * 2 * M1 * M2, G + (size_t)b * N);
        kry::boot_rhs(ctx, G, N, eps_dev, sqrt(cov->tau2), R, nrep);
        kry_embed* e = make_embed_opts(ctx, cov, opts);
        kry::SolveInfo si;
        try {
            kry_embed* pre = make_precond_embed(ctx, cov, opts, e->prec, 1);
            try {
                si = kry::solve(ctx, e, R, p, Wd, p, nrep, opts->rtol, opts->maxit, 0, pre);
            } catch (...) {
                free_embed(pre);
                throw;
            }
            free_embed(pre);
            kry::sigma_to_grid64(ctx, e, Wd, H, nrep, p);
        } catch (...) {
            free_embed(e);
            throw;
        }
        free_embed(e);
        kry::boot_mse(ctx, G, H, N, nrep, cells_dev, ncell, var_dev, bad);
        int* hbad = reinterpret_cast<int*>(ctx->host_pinned);
        KRY_CUDA(cudaMemcpyAsync(hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        KRY_CUDA(cudaStreamSynchronize(ctx->stream));
        if (*hbad) return fail(ctx, KRY_EINVAL, "a target cell index lies outside the grid (its variance is NaN)");
        if (!si.converged) return fail(ctx, KRY_ENOCONV, "CG did not reach rtol for some replicate");
        return KRY_OK;
    });
}

kry_status kry_genhybr_prec(kry_ctx* ctx, const kry_cov* cov, kry_prec prec, int32_t reorth, const double* b_dev,
                            int32_t k, double* x_dev, double* alphas, double* betas, double* z2, double* psi2,
                            double* pl, double* grad, double* psi_dev) {
    return guarded(ctx, [&]() -> kry_status {
        check_cov(cov);
        require_mask(ctx);
        KRY_REQUIRE(prec == KRY_F32 || prec == KRY_F64, KRY_EINVAL, "prec must be KRY_F32 or KRY_F64");
        KRY_REQUIRE(reorth == 0 || reorth == 1, KRY_EINVAL, "reorth must be 0 or 1");
        KRY_REQUIRE(!ctx->sites.active, KRY_EUNSUPPORTED, "genHyBR needs an observation mask (kry_set_mask)");
        KRY_REQUIRE(b_dev != nullptr, KRY_EINVAL, "b_dev must not be NULL");
        KRY_REQUIRE(k >= 1 && k <= 4096, KRY_EINVAL, "k must be in [1, 4096]");
        kry::genhybr_opt(ctx, *cov, prec, reorth != 0, b_dev, k, x_dev, alphas, betas, z2, psi2, pl, grad,
                         psi_dev);
        return KRY_OK;
    });
}

kry_status kry_genhybr(kry_ctx* ctx, const kry_cov* cov, const double* b_dev, int32_t k, double* x_dev,
                       double* alphas, double* betas, double* z2, double* psi2, double* pl, double* grad,
                       double* psi_dev) {
    return kry_genhybr_prec(ctx, cov, KRY_F64, 0, b_dev, k, x_dev, alphas, betas, z2, psi2, pl, grad, psi_dev);
}

kry_status kry_bccb_logdet(kry_ctx* ctx, const kry_cov* cov, double* logdet, double* dlogdet_drange) {
    return guarded(ctx, [&]() -> kry_status {
        check_cov(cov);
        require_mask(ctx);
        KRY_REQUIRE(logdet != nullptr, KRY_EINVAL, "logdet must not be NULL");
        KRY_REQUIRE(2 * (int64_t)ctx->n1 <= KRY_MAX_M && 2 * (int64_t)ctx->n2 <= KRY_MAX_M, KRY_EUNSUPPORTED,
                    "grid too large for the embedding");
        kry::bccb_logdet(ctx, *cov, dlogdet_drange != nullptr, logdet, dlogdet_drange);
        if (!isfinite(*logdet) || (dlogdet_drange && !isfinite(*dlogdet_drange)))
            return fail(ctx, KRY_ENAN, "BCCB log-determinant is NaN/Inf");
        return KRY_OK;
    });
}

}  // extern "C"
