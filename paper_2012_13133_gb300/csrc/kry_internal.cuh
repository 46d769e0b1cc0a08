// Internal declarations of the Kryging CUDA library: context and embedding
// objects, scratch buffers, error handling and launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/kry.h"

// Largest FFT length along one axis and the size of the shared twiddle table
// W[k] = exp(-2 pi i k / KRY_TWN).  Every power-of-two length L <= KRY_TWN
// indexes it with stride KRY_TWN / L.
#define KRY_TWN 8192
#define KRY_MAX_M 8192
#define KRY_MAX_N 4096
#define KRY_MAX_COV 8

// ------------------------------------------------------------------ errors

struct KryError {
    kry_status st;
    std::string msg;
};

#define KRY_CUDA(call)                                                                 \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            throw KryError{KRY_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// Every kernel launch of the library goes through this check, which also
// counts launches (process-wide, for diagnostics).
extern std::atomic<unsigned long long> g_kry_launches;
#define KRY_CHECK_LAUNCH()                                       \
    do {                                                         \
        g_kry_launches.fetch_add(1, std::memory_order_relaxed);  \
        KRY_CUDA(cudaGetLastError());                            \
    } while (0)

// Programmatic dependent launch (sm_90+).  A kernel launched by launch_pdl
// may start while the kernel before it on the stream is still finishing; it
// must call pdl_wait() before it touches anything that kernel writes (the wait
// returns once that grid has completed and its memory is visible; without a
// programmatic predecessor it returns at once).  pdl_launch_dependents() lets
// the next kernel be scheduled as soon as every block of this grid has run it
// (blocks that exit count as having run it), so dependents only fill slots
// this grid no longer needs.  Neither call can wait on anything but the
// predecessor grid's completion.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

#define KRY_REQUIRE(cond, status, text)        \
    do {                                       \
        if (!(cond)) throw KryError{status, text}; \
    } while (0)

// Allow kernel k all the dynamic shared memory the device can give it (the
// opt-in limit minus the kernel's static shared memory).  The limit is a
// process-wide property of the kernel, so it is set once per kernel and device
// to that maximum and never lowered: callers on several threads (server
// slots) with different launch sizes cannot undercut each other's launches.
void kry_allow_max_smem(const void* func);
#define KRY_ALLOW_MAX_SMEM(k) kry_allow_max_smem(reinterpret_cast<const void*>(k))

// Launch kernel k with programmatic stream serialisation (see pdl_wait).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    KRY_CUDA(cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...));
    KRY_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ device buffers

// Device buffer allocated stream-ordered (cudaMallocAsync / cudaFreeAsync on
// its owner's stream), so growing or freeing it never synchronises the device
// and never disturbs a stream capture running in another thread.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaStream_t stream = nullptr;
    void ensure(size_t bytes);   // grows (never shrinks); contents are not kept
    void release();
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// Matvec launch schedule: elements per thread in the row passes and the
// column pass, rows per CTA in the row passes, columns per CTA in the column
// pass (= the column-tile width of the intermediate slab), and the number of
// complex vector pairs per batch.
struct MvSched {
    int ept_row = 8;
    int rows_per_cta = 1;
    int ept_col = 8;
    int cols_per_cta = 4;
    int pairs_per_batch = 0;   // 0 = all pairs at once
    int g16 = 0;               // radix-16 path: rows per block (0 = default)
    int c16 = 0;               // radix-16 path: columns per block / slab tile width (0 = default)
};

struct kry_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;

    // observation pattern
    int n1 = 0, n2 = 0;
    double dx1 = 0, dx2 = 0;
    int64_t p = 0;
    // share of the observed cells whose four grid neighbours are observed too
    // (cells beyond the grid edge count as observed): near 1 for clustered
    // gaps, low for scattered holes; kry_opts.precond = 2 reads it
    double interior = 0.0;
    // FP32 requests run in FP64 for their conditioning (kry_promoted)
    int64_t promoted = 0;
    DevBuf rowptr;   // int32 [n1 + 1]: first observed index of each row
    DevBuf colidx;   // int32 [p]: column of each observed cell
    DevBuf cellidx;  // int32 [p]: row-major cell index of each observed cell

    // shared twiddle tables, W[k] = exp(-2 pi i k / KRY_TWN), and the FP32
    // stage table of the specialised passes (row Ns - 1 + k: W_{16 Ns}^{k m})
    DevBuf tw32, tw64, twt32;
    // FP32 matvecs use the length-specialised passes where they apply (the
    // generic radix-16 passes compute the same transform for the other shapes)
    bool use_spec = true;

    // scratch
    DevBuf slab32, slab64;        // FFT intermediates
    DevBuf work[13];              // Krylov vectors and partials
    DevBuf scal;                  // FP64 Krylov scalars
    DevBuf eig_c, eig_z, eig_d;   // eigenvalue computation (eig_d: derivative eigenvalues)
    DevBuf red;                   // reduction partials
    DevBuf tolbuf, kxbuf;         // CG tolerances, FP64 residual matvec output
    DevBuf cbuf, sbuf;            // kriging-variance right-hand sides and solutions
    DevBuf zbuf, gbuf;            // [y, X] and its solve; kriging grid and weights
    DevBuf boot;                  // bootstrap replicates: fields, predictions, right-hand sides, solves
    DevBuf gk;                    // genGK bases and work vectors
    DevBuf rowptr_full, colidx_full;   // index lists of the whole grid (genGK's and the sites' Sigma matvec)
    int full_n1 = 0, full_n2 = 0;
    // the FFT passes add no nugget (set while the sites' whole-grid Sigma matvec runs)
    bool no_nugget = false;

    // irregular observation sites (kry_set_sites): the Wendland mapping matrix
    // A of Sec. 2 in two forms, by site (the 2 x 2 cells around each site, -1
    // where the weight is zero, and the normalised weights) and by cell (A^T:
    // entries [cellptr[c], cellptr[c + 1]) sorted by site), plus the
    // whole-grid scratch of the site matvec, one buffer per precision (a
    // captured FP32 CG loop keeps its address while FP64 residual matvecs run
    // between its replays)
    struct SiteMap {
        bool active = false;
        DevBuf corner, w64, w32;
        DevBuf cellptr, ent_site, ent_w64, ent_w32, cnt;
        DevBuf grid32, grid64;
    } sites;
    double* host_pinned = nullptr;   // pinned host scratch (4096 doubles)
    int num_sms = 0;
    int max_smem_optin = 0;

    MvSched sched32, sched64;
    // autotuned / user-set schedules keyed by (M1, M2, precision, batch bucket)
    std::map<uint64_t, MvSched> tuned;

    // CUDA-graph capture of the Lanczos loop (a library-owned capture stream
    // joined to the context stream with events)
    bool use_graphs = true;
    cudaStream_t cap_stream = nullptr;

    // optional timing of every matvec (CUDA events on the context stream)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;     // start/stop pairs
    std::vector<int> prof_nvec;
    std::vector<int> prof_dbl;
    double prof_ms_acc[2] = {0.0, 0.0};   // [FP32, FP64] matvec time harvested from replayed graphs
    int64_t prof_calls_acc[2] = {0, 0};
    int64_t prof_vec_acc[2] = {0, 0};
};

struct kry_embed {
    kry_ctx* ctx = nullptr;
    int device = 0;
    int n1 = 0, n2 = 0, M1 = 0, M2 = 0;
    kry_cov cov{};
    kry_prec prec = KRY_F32;
    cudaStream_t stream = nullptr;   // stream of the creating context (stream-ordered frees)
    // eigenvalues transposed to [M2][M1] (column-pass order) and scaled by
    // 1 / (M1 M2), FP64 always and FP32 when prec = KRY_F32
    double* lam64T = nullptr;
    float* lam32T = nullptr;
    // FP32 eigenvalues for the length-specialised column pass: the same
    // [M2][M1] blocks with each column permuted so that the 16 values one
    // thread multiplies (rows t + m M1/16, m < 16) are contiguous at 16 t + m
    // (NULL when that pass does not apply)
    float* lam32P = nullptr;
    double lam_min = 0, lam_max = 0;
    // several covariance settings in one embedding (batched likelihood
    // search): ntheta eigenvalue blocks lam_stride elements apart, per-theta
    // nuggets on the device; a matvec call names how many consecutive real
    // vectors belong to each theta (vectors per theta, even)
    int ntheta = 1;
    int64_t lam_stride = 0;
    double* tau2_dev = nullptr;
};

// ------------------------------------------------------------------ internal entry points

namespace kry {

void init_twiddles(kry_ctx* ctx);

// Release every scratch buffer of ctx (mask, twiddles and schedules stay).
void ctx_trim(kry_ctx* ctx);

// Eigenvalues Lambda = FFT2(c) of the embedding on M1 x M2 (natural order,
// unscaled, FP64) into ctx->eig_c; returns min and max.
void compute_eigs(kry_ctx* ctx, const kry_cov& cov, int n1, int n2, double dx1, double dx2,
                  int M1, int M2, double* lam_min, double* lam_max);

// Matvec passes.  vin/vout: real vectors (T) with leading dimension ld.
// Mode PLAIN: vout = K vin.
template <typename T>
void matvec(kry_ctx* ctx, const kry_embed* e, const T* vin, T* vout, int nvec, int64_t ld,
            double tau2_scale);

// Sigma (no nugget) applied to observed values, evaluated at every grid cell:
// out_grid[n1*n2] per vector (FP64 only; used for kriging).
void sigma_to_grid64(kry_ctx* ctx, const kry_embed* e, const double* vin, double* out_grid, int nvec,
                     int64_t ld, int vpt = 0);

void sample_field(kry_ctx* ctx, const kry_cov& cov, int M1, int M2, const double* xi, double* out);

// Bootstrap helpers (Sec. 3.5): R[b][q] = G[b][cell of q] + tau * eps[b][q];
// var[t] = mean_b (G[b][cells[t]] - H[b][cells[t]])^2 (bad index -> NaN, *bad).
void boot_rhs(kry_ctx* ctx, const double* G, int64_t N, const double* eps, double tau, double* R, int nrep);
void boot_mse(kry_ctx* ctx, const double* G, const double* H, int64_t N, int nrep, const int64_t* cells,
              int64_t ncell, double* var, int* bad);

// Irregular sites (sites.cu, Sec. 2 Wendland mapping A): build ctx->sites for
// nsite device coordinate pairs (false if a site lies outside the domain);
// grid[v] = scale[v] A^T vin[v] on the whole grid; vout[v] = A grid[v] + tau2
// scale[v] vin[v] with per-block partials of (scale[v] vin[v])^T vout[v]
// (site_num_partials() blocks when dots is NULL, nds otherwise).
bool build_sites(kry_ctx* ctx, int n1, int n2, double dx1, double dx2, const double* sites, int64_t nsite);
int site_num_partials(kry_ctx* ctx);
template <typename T>
void site_scatter(kry_ctx* ctx, const T* vin, int64_t ld_in, const double* scale, int nvec, T* grid, const int* skip);
template <typename T>
void site_gather(kry_ctx* ctx, const T* grid, const T* vin, int64_t ld_in, const double* scale, T* vout,
                 int64_t ld_out, int nvec, double tau2, const double* tau2v, int vpt, double* dots, int nds,
                 const int* skip);

// Replace the eigenvalues Lambda in ctx->eig_c (natural order, unscaled) by
// 1 / (max(Lambda, 0) + tau2): the torus inverse (S + tau2 I)^-1.
void invert_eigs(kry_ctx* ctx, int M1, int M2, double tau2);

// Overwrite FP64 embedding e's eigenvalues with those of d Sigma / d(range).
void drange_embedding(kry_ctx* ctx, const kry_cov& cov, kry_embed* e);

// Embedding of one covariance setting on the mask's grid (library-owned).
kry_embed* make_embed_internal(kry_ctx* ctx, const kry_cov* cov, kry_prec prec);
void free_embed_internal(kry_embed* e);

// genHyBR with k genGK steps (Sec. 3.2, Alg. 1; Eq. prof_lik): b = y - X beta on the
// observed cells; x_out (whole grid, may be NULL), alphas/betas[k+1] (host, may be NULL).
// prec KRY_F32: FP32 Krylov vectors and matvec, FP64 scalars and reductions.
void genhybr(kry_ctx* ctx, const kry_cov& cov, kry_prec prec, const double* b, int k, double* x_out, double* alphas,
             double* betas, double* z2, double* psi2, double* pl, double* grad = nullptr, double* psi_out = nullptr);

// BCCB approximation of log det Sigma (no nugget) on the mask's grid and, if
// deriv, of its range derivative (Sec. 3.3, Appendix A).
void bccb_logdet(kry_ctx* ctx, const kry_cov& cov, bool deriv, double* logdet, double* dlogdet);

int smem_limit(kry_ctx* ctx);

// Record a profiling event on the context stream; inside a stream capture it
// becomes an external event-record node, so it still times the graph replay.
void prof_record(kry_ctx* ctx, cudaEvent_t ev);

// Schedule key and lookup (falls back to the per-precision default).
uint64_t sched_key(int M1, int M2, bool dbl, int nvec);
const MvSched& sched_for(kry_ctx* ctx, int M1, int M2, bool dbl, int nvec);

struct SolveInfo {
    int iters = 0;
    double relres = 0.0;
    bool converged = false;
};

struct GlsResult {
    double loglik, quad;
    double beta[KRY_MAX_COV];
    bool ok;
};

}  // namespace kry
