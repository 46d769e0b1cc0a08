// Krylov loops on the covariance matvec:
//   * stochastic Lanczos quadrature for log det K (Sec. 3.3 names stochastic
//     trace estimation as the alternative to the circulant log-det);
//   * conjugate gradients for K X = B with FP64 residual replacement (the
//     matvec-only solves that replace the O(n^3) inversions of Sec. 3);
//   * GLS beta and the profile log-likelihood; kriging means (the paper's
//     x-hat, Eq. act_xhat, by Woodbury) and simple-kriging variances (the
//     quantity the bootstrap of Sec. 3.5 estimates).
//
// Vectors are FP32 (or FP64 for FP64 embeddings); every dot product is
// accumulated in FP64 per block and reduced in a fixed order by one small
// kernel, so results do not depend on scheduling.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dfloat.cuh"
#include "fft.cuh"
#include "kry_internal.cuh"
#include "matern.cuh"

namespace kry {

template <typename T>
void matvec_ex(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
               int64_t ld_out, int nvec, double* dots, int nds, int vpt = 0, const int* skip = nullptr);
int matvec_num_partials(kry_ctx* ctx, const kry_embed* e, bool dbl, int nvec);

static const int RED_BLOCKS = 128;   // fixed block count of the vector reductions

// ------------------------------------------------------------------ probes

// splitmix64 output function (Steele, Lea & Flood 2014) of state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Vector v holds Rademacher probe (v mod nprobe): every covariance setting of a
// batched search sees the same probes.
template <typename T>
__global__ void k_probes(T* __restrict__ W, int64_t p, int nprobe, uint64_t seed) {
    const int v = blockIdx.y;
    const uint64_t k = (uint64_t)(v % nprobe);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t key = seed ^ ((k << 32) | (uint64_t)i);
        W[(int64_t)v * p + i] = (splitmix64(key) >> 63) ? (T)-1 : (T)1;
    }
}

// Run fn() under stream capture on the library's capture stream and replay the
// captured graph once, ordered after earlier work on ctx->stream and before
// later work on it.  Without graphs (ctx->use_graphs false) fn() runs directly.
template <class F>
static void run_captured(kry_ctx* ctx, F&& fn) {
    if (!ctx->use_graphs) {
        fn();
        return;
    }
    if (!ctx->cap_stream) KRY_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = ctx->stream, cap = ctx->cap_stream;
    cudaEvent_t fork, join;
    KRY_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    KRY_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    KRY_CUDA(cudaEventRecord(fork, user));
    KRY_CUDA(cudaStreamWaitEvent(cap, fork, 0));
    cudaGraph_t graph = nullptr;
    ctx->stream = cap;
    KRY_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    try {
        fn();
    } catch (...) {
        cudaStreamEndCapture(cap, &graph);
        if (graph) cudaGraphDestroy(graph);
        ctx->stream = user;
        cudaEventDestroy(fork);
        cudaEventDestroy(join);
        throw;
    }
    ctx->stream = user;
    KRY_CUDA(cudaStreamEndCapture(cap, &graph));
    cudaGraphExec_t exec = nullptr;
    KRY_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    KRY_CUDA(cudaGraphLaunch(exec, cap));
    KRY_CUDA(cudaEventRecord(join, cap));
    KRY_CUDA(cudaStreamWaitEvent(user, join, 0));
    KRY_CUDA(cudaGraphExecDestroy(exec));
    KRY_CUDA(cudaGraphDestroy(graph));
    KRY_CUDA(cudaEventDestroy(fork));
    KRY_CUDA(cudaEventDestroy(join));
}

// A launch sequence captured once into a CUDA graph (on the library's capture
// stream) and replayed on ctx->stream as often as needed.  Replays add the
// captured kernel count to the launch counter.  With profiling on, the matvec
// event pairs recorded during capture are re-recorded by every replay; the
// caller synchronises the stream after a replay and calls harvest(), which adds
// their times to the context's totals.
struct Replay {
    kry_ctx* ctx = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;
    std::vector<cudaEvent_t> ev;   // start/stop pairs owned by the graph's profiling nodes
    std::vector<int> nvec, dbl;
    explicit Replay(kry_ctx* c) : ctx(c) {}
    Replay(const Replay&) = delete;
    Replay& operator=(const Replay&) = delete;
    ~Replay() {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    template <class F>
    void capture(F&& fn) {
        if (!ctx->cap_stream) KRY_CUDA(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = ctx->stream, cap = ctx->cap_stream;
        const unsigned long long n0 = g_kry_launches.load();
        const size_t p0 = ctx->prof_nvec.size();
        cudaGraph_t graph = nullptr;
        ctx->stream = cap;
        KRY_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
        try {
            fn();
        } catch (...) {
            cudaStreamEndCapture(cap, &graph);
            if (graph) cudaGraphDestroy(graph);
            ctx->stream = user;
            throw;
        }
        ctx->stream = user;
        // the profiling pairs recorded by the capture belong to the graph from now on
        ev.assign(ctx->prof_ev.begin() + 2 * p0, ctx->prof_ev.end());
        nvec.assign(ctx->prof_nvec.begin() + p0, ctx->prof_nvec.end());
        dbl.assign(ctx->prof_dbl.begin() + p0, ctx->prof_dbl.end());
        ctx->prof_ev.resize(2 * p0);
        ctx->prof_nvec.resize(p0);
        ctx->prof_dbl.resize(p0);
        KRY_CUDA(cudaStreamEndCapture(cap, &graph));
        const cudaError_t err = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        KRY_CUDA(err);
        kernels = g_kry_launches.load() - n0;
        g_kry_launches.fetch_sub(kernels);   // counted when replayed
    }
    void launch() {
        KRY_CUDA(cudaGraphLaunch(exec, ctx->stream));
        g_kry_launches.fetch_add(kernels);
    }
    // After the stream has been synchronised following launch().
    void harvest() {
        for (size_t i = 0; i < nvec.size(); ++i) {
            float t = 0.f;
            KRY_CUDA(cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
            ctx->prof_ms_acc[dbl[i]] += t;
            ctx->prof_calls_acc[dbl[i]] += 1;
            ctx->prof_vec_acc[dbl[i]] += nvec[i];
        }
    }
};

// ------------------------------------------------------------------ block reduction helper

template <int N>
__device__ __forceinline__ void block_sum_store(double (&v)[N], double* out, int64_t out_stride) {
    __shared__ double red[N][32];
#pragma unroll
    for (int a = 0; a < N; ++a)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int a = 0; a < N; ++a) red[a][w] = v[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int a = 0; a < N; ++a) {
            double s = 0.0;
            for (int k = 0; k < nw; ++k) s += red[a][k];
            out[a * out_stride] = s;
        }
    }
}

// Sum of part[0..n) by one block in a fixed order (strided per-thread sums,
// then a shuffle tree, then the warp sums in order); the result is valid in
// thread 0.  Deterministic for a given block size.
__device__ __forceinline__ double block_sum(const double* __restrict__ part, int n) {
    __shared__ double ws[32];
    double v = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) v += part[b];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    return t;
}

static const int FIN_THREADS = 256;   // block size of the per-vector finalisers

// VW consecutive elements of type T through one 16-byte access (VW = 16 /
// sizeof(T)), or one element (VW = 1).  The caller guarantees alignment.
template <typename T, int VW>
__device__ __forceinline__ void load_vec(const T* __restrict__ src, T (&out)[VW]) {
    if constexpr (VW * sizeof(T) == 16) {
        const int4 q = *reinterpret_cast<const int4*>(src);
        memcpy(out, &q, 16);
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) out[e] = src[e];
    }
}

template <typename T, int VW>
__device__ __forceinline__ void store_vec(T* __restrict__ dst, const T (&in)[VW]) {
    if constexpr (VW * sizeof(T) == 16) {
        int4 q;
        memcpy(&q, in, 16);
        *reinterpret_cast<int4*>(dst) = q;
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) dst[e] = in[e];
    }
}

// VW elements of the reorthogonalisation store as T: the store is T itself,
// or FP16 (VW = 4: one 8-byte access).
template <typename T, typename Sq, int VW>
__device__ __forceinline__ void load_as(const Sq* __restrict__ src, T (&out)[VW]) {
    if constexpr (std::is_same<Sq, T>::value) {
        load_vec<T, VW>(src, out);
    } else if constexpr (VW == 4) {
        const uint2 q = *reinterpret_cast<const uint2*>(src);
        __half2 h[2];
        memcpy(h, &q, 8);
        const float2 a = __half22float2(h[0]), b = __half22float2(h[1]);
        out[0] = (T)a.x;
        out[1] = (T)a.y;
        out[2] = (T)b.x;
        out[3] = (T)b.y;
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) out[e] = (T)__half2float(src[e]);
    }
}

// ------------------------------------------------------------------ Lanczos

#define KRY_MAX_STEPS 256

struct LanczosState {
    double* s_cur;    // [nprobe] scale of the current vector: q_j = s_cur * W_cur
    double* s_prev;   // [nprobe]
    double* alpha;    // [nprobe][nsteps]
    double* beta;     // [nprobe][nsteps]
    int* m_eff;       // [nprobe] Lanczos steps kept (early stop on breakdown)
    // partial reorthogonalisation only (all NULL without it)
    double* s_hist;   // [nprobe][nsteps] scale of every stored basis vector: q_i = s_hist[i] * W_i
    double* omega;    // [3][nprobe][nsteps + 1] estimates of q_j^T q_k for j-1, j, j+1 (buffer j mod 3)
    double* coef;     // [nprobe][nsteps] s_i * q_i^T w of the vector being reorthogonalised
    int* flag;        // [nprobe] 1: reorthogonalise the new vector of this step
    int* force;       // [nprobe] 1: the next new vector is reorthogonalised too
    double* pre2;     // [nprobe] ||w||^2 before the Gram-Schmidt pass of a flagged vector
};

__global__ void k_lanczos_init(LanczosState S, int nprobe, int nsteps, double s0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprobe) return;
    S.s_cur[k] = s0;
    S.s_prev[k] = 0.0;
    S.m_eff[k] = nsteps;
    if (S.s_hist) {
        S.s_hist[(int64_t)k * nsteps] = s0;
        S.omega[(int64_t)k * (nsteps + 1)] = 1.0;   // omega_{0,0}
        S.flag[k] = 0;
        S.force[k] = 0;
    }
}

// alpha_j = sum of the block partials of q_j^T K q_j (fixed order).
__global__ void k_lanczos_alpha(LanczosState S, const double* __restrict__ part, int nblk, int nprobe, int nsteps,
                                int j) {
    const int k = blockIdx.x;   // one block per vector
    const double a = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x == 0) S.alpha[(int64_t)k * nsteps + j] = a;
}

// w_next = U - alpha_j s_cur W_cur - beta_{j-1} s_prev W_prev;  partial ||w_next||^2.
// VW elements per access when every vector start is 16-byte aligned.
template <typename T, int VW>
__global__ void k_lanczos_update(const T* __restrict__ U, const T* __restrict__ Wc, const T* __restrict__ Wp,
                                 T* __restrict__ Wn, int64_t p, LanczosState S, int nsteps, int j,
                                 double* __restrict__ part) {
    const int k = blockIdx.y;
    const double a = S.alpha[(int64_t)k * nsteps + j];
    const T ca = (T)(a * S.s_cur[k]);
    const T cb = (T)((j > 0 ? S.beta[(int64_t)k * nsteps + j - 1] : 0.0) * S.s_prev[k]);
    const int64_t off = (int64_t)k * p;
    const int64_t nv = p / VW;
    DotAcc<T> nrm;
    for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv; xv += (int64_t)gridDim.x * blockDim.x) {
        T u[VW], wc[VW], wp[VW];
        load_vec<T, VW>(U + off + xv * VW, u);
        load_vec<T, VW>(Wc + off + xv * VW, wc);
        // at j = 0 there is no previous vector (its buffer is not initialised)
        if (j > 0) {
            load_vec<T, VW>(Wp + off + xv * VW, wp);
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) wp[e] = (T)0;
        }
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            u[e] = u[e] - ca * wc[e] - cb * wp[e];
            nrm.add_prod(u[e], u[e]);
        }
        store_vec<T, VW>(Wn + off + xv * VW, u);
    }
    double acc[1] = {nrm.value()};
    block_sum_store<1>(acc, part + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

// beta_j = ||w_next||; early stop when beta_j < 1e-12 |alpha_1|; rescale.
__global__ void k_lanczos_beta(LanczosState S, const double* __restrict__ part, int nblk, int nprobe, int nsteps,
                               int j) {
    const int k = blockIdx.x;   // one block per vector
    const double s = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x != 0) return;
    const double bj = sqrt(s);
    const bool stopped = S.m_eff[k] < nsteps;
    if (!stopped && bj < 1e-12 * fabs(S.alpha[(int64_t)k * nsteps])) S.m_eff[k] = j + 1;
    const bool now_stopped = S.m_eff[k] < nsteps;
    S.beta[(int64_t)k * nsteps + j] = now_stopped ? 0.0 : bj;
    S.s_prev[k] = S.s_cur[k];
    S.s_cur[k] = now_stopped ? 0.0 : 1.0 / bj;
    if (S.s_hist && j + 1 < nsteps) S.s_hist[(int64_t)k * nsteps + j + 1] = S.s_cur[k];
}

// ------------------------------------------------------------------ partial reorthogonalisation
//
// The basis may lose orthogonality (Sec. 3.2, which leaves a reorthogonalisation
// scheme to the user); in FP32 the loss reaches the Gauss quadrature within a
// few tens of steps.  Partial reorthogonalisation (H. D. Simon, "The Lanczos
// algorithm with partial reorthogonalization", Math. Comp. 42, 1984) tracks
// estimates omega_{j,k} of q_j^T q_k by a scalar recurrence derived from the
// three-term recurrences of q_j and q_k, with a rounding term of size
// eps_round (beta_k + beta_j); when the largest estimate for the new vector
// exceeds sqrt(eps) (eps = unit roundoff of the vectors), the new vector and
// the one after it are orthogonalised against every stored basis vector
// (classical Gram-Schmidt, repeated once when it cancels most of the vector)
// and their estimates reset to what the pass leaves: eps, or for FP32 vectors,
// whose basis is stored in FP16 (2^-11 relative rounding, half the traffic of
// an FP32 store), the FP16 rounding of a removed component of size sqrt(eps),
// about 2 eps.  The rounding term uses
// eps_round = eps log2(M1 M2): the local error of a step is that of the FFT
// matvec, which grows with the log of the transform size.  With eps alone,
// FP32 runs on smooth long-range covariances (512^2 grid, range >= 0.1)
// lost orthogonality unnoticed: per-probe values up to 3% off the FP64 run,
// some NaN; with eps_round they agree to 2e-5 at 5% more time.  Semi-orthogonality
// (|q_j^T q_k| <= sqrt(eps)) keeps the tridiagonal equal to the projection of K
// on the Krylov space up to O(eps ||K||) (Simon 1984).  Decisions are per
// vector, on the device, so the launch sequence is fixed and graph-capturable.

// Estimates for q_{j+1} from ||w||^2 partials (before any reorthogonalisation);
// sets flag[k] when w is to be reorthogonalised.
__global__ void k_pro_omega(LanczosState S, const double* __restrict__ part, int nblk, int nsteps, int j,
                            double eps, double eps_round, double omega_reset) {
    const int k = blockIdx.x;   // one block per vector
    const double s = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x != 0) return;
    const int64_t ostride = (int64_t)gridDim.x * (nsteps + 1);
    double* on = S.omega + ((j + 1) % 3) * ostride + (int64_t)k * (nsteps + 1);   // omega_{j+1, .}
    const double* oc = S.omega + (j % 3) * ostride + (int64_t)k * (nsteps + 1);   // omega_{j, .}
    const double* op = S.omega + ((j + 2) % 3) * ostride + (int64_t)k * (nsteps + 1);   // omega_{j-1, .}
    const double* al = S.alpha + (int64_t)k * nsteps;
    const double* be = S.beta + (int64_t)k * nsteps;
    const double bj = sqrt(s);
    if (S.m_eff[k] < nsteps || !(bj > 0.0)) {   // stopped: nothing to keep orthogonal
        S.flag[k] = 0;
        return;
    }
    const double aj = al[j];
    double tnorm = fabs(aj) + bj;
    for (int i = 0; i < j; ++i) tnorm = fmax(tnorm, fabs(al[i]) + be[i]);
    double worst = 0.0;
    for (int i = 0; i < j; ++i) {
        double t = be[i] * oc[i + 1] + (al[i] - aj) * oc[i] - be[j - 1] * op[i];
        if (i > 0) t += be[i - 1] * oc[i - 1];
        t += copysign(eps_round * (be[i] + bj), t);
        on[i] = t / bj;
        worst = fmax(worst, fabs(on[i]));
    }
    on[j] = eps_round * tnorm / bj;
    on[j + 1] = 1.0;
    worst = fmax(worst, fabs(on[j]));
    const int f = (S.force[k] || worst > sqrt(eps)) ? 1 : 0;
    S.flag[k] = f;
    S.pre2[k] = s;
    S.force[k] = f && !S.force[k];   // the vector after a reorthogonalised one is reorthogonalised too
    if (f)
        for (int i = 0; i <= j; ++i) on[i] = omega_reset;
}

// "Twice is enough" (Kahan; Parlett, The Symmetric Eigenvalue Problem, 1980,
// Sec. 6-9): a flagged vector whose norm fell below 1/sqrt(2) of its norm
// before the Gram-Schmidt pass lost most of itself to cancellation, and its
// rounding errors are then large relative to what is left; it stays flagged
// for a second pass, every other vector is unflagged.
__global__ void k_reorth_again(LanczosState S, const double* __restrict__ part, int nblk) {
    const int k = blockIdx.x;   // one block per vector
    if (!S.flag[k]) return;
    const double s = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x != 0) return;
    S.flag[k] = (s < 0.5 * S.pre2[k]) ? 1 : 0;
    S.pre2[k] = s;
}

// Partial dot products W_i^T w (i = 0..j) of each flagged vector against the
// basis store Q (T, or FP16 for FP32 vectors), 8 basis vectors per sweep over
// the block's slice of w, VW elements per access.  Products and per-thread sums
// are in the vector precision T (a coefficient only needs a few correct digits:
// it removes a component of size <= sqrt(eps)), the block sums in FP64.  dpart rows are [nvec][nsteps + 8][nblk]: a sweep's rows
// past j (zeros) stay in the vector's padding.
template <typename T, typename Sq, int VW>
__global__ void k_reorth_dots(const Sq* __restrict__ Q, const T* __restrict__ Wn, int nvec, int64_t p, int j,
                              const int* __restrict__ flag, int nsteps, double* __restrict__ dpart) {
    const int k = blockIdx.y;
    if (!flag[k]) return;
    const T* w = Wn + (int64_t)k * p;
    const int64_t nv = p / VW;
    for (int i0 = 0; i0 <= j; i0 += 8) {
        T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv;
             xv += (int64_t)gridDim.x * blockDim.x) {
            T wv[VW];
            load_vec<T, VW>(w + xv * VW, wv);
#pragma unroll
            for (int a = 0; a < 8; ++a)
                if (i0 + a <= j) {
                    T qv[VW];
                    load_as<T, Sq, VW>(Q + ((int64_t)(i0 + a) * nvec + k) * p + xv * VW, qv);
#pragma unroll
                    for (int e = 0; e < VW; ++e) acc[a] += qv[e] * wv[e];
                }
        }
        double accd[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) accd[a] = (double)acc[a];
        block_sum_store<8>(accd, dpart + ((int64_t)k * (nsteps + 8) + i0) * gridDim.x + blockIdx.x, gridDim.x);
        __syncthreads();
    }
}

// coef_i = s_i (q_i^T w) = s_i^2 (W_i^T w) for a store of the unnormalised W_i,
// or (q_i^T w) / sqrt(p) = (H_i^T w) / p for the FP16 store H_i = sqrt(p) q_i
// (hscale = 1 / p, else 0), summed over the partials in a fixed order.
__global__ void k_reorth_coef(LanczosState S, const double* __restrict__ dpart, int nblk, int nsteps, int j,
                              double hscale) {
    const int k = blockIdx.x;
    if (!S.flag[k]) return;
    for (int i = 0; i <= j; ++i) {
        const double d = block_sum(dpart + ((int64_t)k * (nsteps + 8) + i) * nblk, nblk);
        if (threadIdx.x == 0) {
            const double si = S.s_hist[(int64_t)k * nsteps + i];
            S.coef[(int64_t)k * nsteps + i] = hscale > 0.0 ? hscale * d : si * si * d;
        }
        __syncthreads();
    }
}

// H = FP16(sqrt(p) s_k W_k) for every vector k: the new basis vector,
// normalised and scaled to entries of order one, for the reorthogonalisation
// store.
template <int VW>
__global__ void k_store_half(const float* __restrict__ W, const double* __restrict__ s, double sqrtp,
                             __half* __restrict__ H, int64_t p) {
    const int k = blockIdx.y;
    const float sc = (float)(s[k] * sqrtp);
    const int64_t off = (int64_t)k * p;
    const int64_t nv = p / VW;
    for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv; xv += (int64_t)gridDim.x * blockDim.x) {
        float w[VW];
        load_vec<float, VW>(W + off + xv * VW, w);
        if constexpr (VW == 4) {
            __half2 h[2] = {__floats2half2_rn(sc * w[0], sc * w[1]), __floats2half2_rn(sc * w[2], sc * w[3])};
            uint2 q;
            memcpy(&q, h, 8);
            *reinterpret_cast<uint2*>(H + off + xv * VW) = q;
        } else {
#pragma unroll
            for (int e = 0; e < VW; ++e) H[off + xv * VW + e] = __float2half_rn(sc * w[e]);
        }
    }
}

// w -= sum_i coef_i W_i (in the basis precision) for flagged vectors, VW
// elements per access; partial ||w||^2 replaces the update's so that beta_j is
// the norm after reorthogonalisation.
template <typename T, typename Sq, int VW>
__global__ void k_reorth_apply(const Sq* __restrict__ Q, T* __restrict__ Wn, int nvec, int64_t p, int j,
                               LanczosState S, int nsteps, double* __restrict__ part) {
    const int k = blockIdx.y;
    if (!S.flag[k]) return;
    __shared__ T c[KRY_MAX_STEPS];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) c[i] = (T)S.coef[(int64_t)k * nsteps + i];
    __syncthreads();
    T* w = Wn + (int64_t)k * p;
    const int64_t nv = p / VW;
    DotAcc<T> nrm;
    for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv; xv += (int64_t)gridDim.x * blockDim.x) {
        T proj[VW];
#pragma unroll
        for (int e = 0; e < VW; ++e) proj[e] = 0;
#pragma unroll 4
        for (int i = 0; i <= j; ++i) {
            T qv[VW];
            load_as<T, Sq, VW>(Q + ((int64_t)i * nvec + k) * p + xv * VW, qv);
#pragma unroll
            for (int e = 0; e < VW; ++e) proj[e] += c[i] * qv[e];
        }
        T r[VW];
        load_vec<T, VW>(w + xv * VW, r);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            r[e] -= proj[e];
            nrm.add_prod(r[e], r[e]);
        }
        store_vec<T, VW>(w + xv * VW, r);
    }
    double acc[1] = {nrm.value()};
    block_sum_store<1>(acc, part + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

// Gauss quadrature of z^T log(K) z from the Lanczos tridiagonal: implicit QL
// iterations with Wilkinson shifts, the published procedure tql2 (Bowdler,
// Martin, Reinsch & Wilkinson, "The QR and QL algorithms for symmetric
// matrices", Numer. Math. 1968; EISPACK's tql2), rotating only the first row of
// the eigenvector matrix (Golub & Welsch 1969).
//
// K = sigma2 A Sigma A^T + tau2 I has every eigenvalue >= tau2, and so has
// every Ritz value of exact arithmetic.  Rounding in the matvec can move the
// smallest computed Ritz values below that bound (to zero or below once it is
// of the order of tau2, where the log would be undefined), so the nodes are
// taken as max(d_i, tau2) of the vector's setting (tau2v[v / vpt] for a
// batched embedding, tau2 otherwise).
__global__ void k_quadrature(const LanczosState S, int nprobe, int nsteps, double znorm2, double* __restrict__ out,
                             double tau2, const double* __restrict__ tau2v, int vpt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprobe) return;
    const double lb = (tau2v && vpt > 0) ? tau2v[k / vpt] : tau2;
    const int n = S.m_eff[k];
    double d[KRY_MAX_STEPS], e[KRY_MAX_STEPS], z[KRY_MAX_STEPS];
    for (int i = 0; i < n; ++i) {
        d[i] = S.alpha[(int64_t)k * nsteps + i];
        e[i] = (i < n - 1) ? S.beta[(int64_t)k * nsteps + i] : 0.0;
        z[i] = (i == 0) ? 1.0 : 0.0;
    }
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < n; ++l) {
        for (int iter = 0; iter < 100; ++iter) {
            int m = l;
            for (; m < n - 1; ++m) {
                const double dd = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= eps * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, pp = 0.0;
            bool deflated = false;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i];
                const double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= pp;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                const double zf = z[i + 1];
                z[i + 1] = s * z[i] + c * zf;
                z[i] = c * z[i] - s * zf;
            }
            if (deflated) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc += z[i] * z[i] * log(fmax(d[i], lb));
    out[k] = znorm2 * acc;
}

// Lanczos over nvec vectors (vector v holds probe v mod nprobe; vpt consecutive
// vectors share one covariance setting of a batched embedding, 0 = one
// setting).  Step 0 runs directly (it sizes every buffer); steps 1.. are
// captured into one CUDA graph and replayed as one launch.  Without
// reorthogonalisation three basis vectors rotate through three buffers; with it
// every basis vector is kept ([nsteps][nvec][p]) for the Gram-Schmidt passes.
template <typename T>
static void lanczos_logdet(kry_ctx* ctx, const kry_embed* e, int nvec, int nprobe, int nsteps, uint64_t seed,
                           double* per_vec, int vpt, bool reorth) {
    const bool dbl = sizeof(T) == 8;
    const int64_t p = ctx->p;
    const int nblkC = matvec_num_partials(ctx, e, dbl, nvec);
    const size_t vbytes = (size_t)nvec * p * sizeof(T);
    ctx->work[0].ensure(vbytes);
    T* U = ctx->work[0].as<T>();
    T* Q = nullptr;   // FP64 basis store with reorthogonalisation
    T* W[3] = {nullptr, nullptr, nullptr};
    // FP32 with reorthogonalisation: the three-term recurrence runs on three
    // rotating FP32 vectors, and every basis vector is also kept, normalised,
    // in an FP16 store for the Gram-Schmidt passes (half the traffic and memory
    // of an FP32 store; k_store_half)
    const bool hstore = reorth && !dbl;
    __half* H = nullptr;
    if (reorth && dbl) {
        ctx->work[1].ensure(vbytes * nsteps);
        Q = ctx->work[1].as<T>();
    } else if (hstore) {
        ctx->work[1].ensure((size_t)nvec * p * sizeof(__half) * nsteps);
        H = ctx->work[1].as<__half>();
        ctx->work[2].ensure(3 * vbytes);
        for (int b = 0; b < 3; ++b) W[b] = ctx->work[2].as<T>() + (size_t)b * nvec * p;
    } else {
        for (int b = 1; b < 4; ++b) ctx->work[b].ensure(vbytes);
        for (int b = 0; b < 3; ++b) W[b] = ctx->work[b + 1].as<T>();
    }
    auto basis = [&](int i) -> T* { return Q ? Q + (size_t)i * nvec * p : W[i % 3]; };
    const int nred = std::max(nblkC, RED_BLOCKS);
    ctx->work[4].ensure((size_t)nvec * nred * sizeof(double));
    double* part = ctx->work[4].as<double>();
    const size_t nsc = (size_t)nvec * (2 * nsteps + 4) + nvec;
    const size_t npro = reorth ? (size_t)nvec * (2 * nsteps + 3 * (nsteps + 1) + 1) : 0;
    ctx->scal.ensure((nsc + npro) * sizeof(double));
    double* sc = ctx->scal.as<double>();
    LanczosState S;
    S.s_cur = sc;
    S.s_prev = sc + nvec;
    S.alpha = sc + 2 * nvec;
    S.beta = S.alpha + (size_t)nvec * nsteps;
    double* res = S.beta + (size_t)nvec * nsteps;
    ctx->work[5].ensure((size_t)nvec * 3 * sizeof(int));
    S.m_eff = ctx->work[5].as<int>();
    S.s_hist = S.omega = S.coef = S.pre2 = nullptr;
    S.flag = S.force = nullptr;
    double* dpart = nullptr;
    if (reorth) {
        S.s_hist = sc + nsc;
        S.coef = S.s_hist + (size_t)nvec * nsteps;
        S.omega = S.coef + (size_t)nvec * nsteps;
        S.pre2 = S.omega + (size_t)3 * nvec * (nsteps + 1);
        S.flag = S.m_eff + nvec;
        S.force = S.flag + nvec;
        ctx->work[6].ensure((size_t)nvec * (nsteps + 8) * RED_BLOCKS * sizeof(double));
        dpart = ctx->work[6].as<double>();
    }
    const double eps = dbl ? 1.1102230246251565e-16 : 5.9604644775390625e-08;   // unit roundoff of T
    // rounding term of the omega recurrence: the local error of one Lanczos step
    // is dominated by the FFT matvec, whose error grows like log2 of the
    // transform size (eps log2(M1 M2) ||K||, not eps ||K||)
    const double eps_round = eps * std::log2((double)e->M1 * (double)e->M2);
    // what a Gram-Schmidt pass leaves of q_i^T w: rounding of order eps, or, with
    // the FP16 store, the FP16 rounding (2^-11) of a removed component of size
    // up to sqrt(eps)
    const double omega_reset = hstore ? std::max(eps, std::sqrt(eps) * 4.8828125e-4) : eps;

    const int tb = 256;
    k_lanczos_init<<<(nvec + tb - 1) / tb, tb, 0, ctx->stream>>>(S, nvec, nsteps, 1.0 / sqrt((double)p));
    KRY_CHECK_LAUNCH();
    dim3 gp((unsigned)std::min<int64_t>((p + 255) / 256, 1024), nvec);
    k_probes<T><<<gp, 256, 0, ctx->stream>>>(basis(0), p, nprobe, seed);
    KRY_CHECK_LAUNCH();
    constexpr int VW = 16 / sizeof(T);   // 16-byte accesses when every vector start is 16-byte aligned
    const dim3 gu(RED_BLOCKS, nvec);
    const double sqrtp = sqrt((double)p);
    auto store_half = [&](int i) {   // H_i from basis(i) and its scale s_cur
        if constexpr (sizeof(T) == 4) {
            if (p % VW == 0)
                k_store_half<VW><<<gu, 256, 0, ctx->stream>>>(basis(i), S.s_cur, sqrtp, H + (size_t)i * nvec * p, p);
            else
                k_store_half<1><<<gu, 256, 0, ctx->stream>>>(basis(i), S.s_cur, sqrtp, H + (size_t)i * nvec * p, p);
            KRY_CHECK_LAUNCH();
        }
    };
    // Gram-Schmidt dot products and update against the basis store
    auto reorth_dots = [&](T* Wn, int j) {
        if constexpr (sizeof(T) == 4) {
            if (p % VW == 0)
                k_reorth_dots<T, __half, VW><<<gu, 256, 0, ctx->stream>>>(H, Wn, nvec, p, j, S.flag, nsteps, dpart);
            else
                k_reorth_dots<T, __half, 1><<<gu, 256, 0, ctx->stream>>>(H, Wn, nvec, p, j, S.flag, nsteps, dpart);
        } else {
            if (p % VW == 0)
                k_reorth_dots<T, T, VW><<<gu, 256, 0, ctx->stream>>>(Q, Wn, nvec, p, j, S.flag, nsteps, dpart);
            else
                k_reorth_dots<T, T, 1><<<gu, 256, 0, ctx->stream>>>(Q, Wn, nvec, p, j, S.flag, nsteps, dpart);
        }
        KRY_CHECK_LAUNCH();
    };
    auto reorth_apply = [&](T* Wn, int j) {
        if constexpr (sizeof(T) == 4) {
            if (p % VW == 0)
                k_reorth_apply<T, __half, VW><<<gu, 256, 0, ctx->stream>>>(H, Wn, nvec, p, j, S, nsteps, part);
            else
                k_reorth_apply<T, __half, 1><<<gu, 256, 0, ctx->stream>>>(H, Wn, nvec, p, j, S, nsteps, part);
        } else {
            if (p % VW == 0)
                k_reorth_apply<T, T, VW><<<gu, 256, 0, ctx->stream>>>(Q, Wn, nvec, p, j, S, nsteps, part);
            else
                k_reorth_apply<T, T, 1><<<gu, 256, 0, ctx->stream>>>(Q, Wn, nvec, p, j, S, nsteps, part);
        }
        KRY_CHECK_LAUNCH();
    };
    if (hstore) store_half(0);
    auto step = [&](int j) {
        cudaStream_t st = ctx->stream;
        T* Wc = basis(j);
        T* Wp = basis(j > 0 ? j - 1 : 0);
        matvec_ex<T>(ctx, e, Wc, p, S.s_cur, U, p, nvec, part, nblkC, vpt);
        k_lanczos_alpha<<<nvec, FIN_THREADS, 0, st>>>(S, part, nblkC, nvec, nsteps, j);
        KRY_CHECK_LAUNCH();
        if (j == nsteps - 1) return;
        T* Wn = basis(j + 1);
        if (p % VW == 0)
            k_lanczos_update<T, VW><<<gu, 256, 0, st>>>(U, Wc, Wp, Wn, p, S, nsteps, j, part);
        else
            k_lanczos_update<T, 1><<<gu, 256, 0, st>>>(U, Wc, Wp, Wn, p, S, nsteps, j, part);
        KRY_CHECK_LAUNCH();
        if (reorth) {
            k_pro_omega<<<nvec, FIN_THREADS, 0, st>>>(S, part, RED_BLOCKS, nsteps, j, eps, eps_round, omega_reset);
            KRY_CHECK_LAUNCH();
            reorth_dots(Wn, j);
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) {
                    // second Gram-Schmidt pass for vectors that lost most of their norm
                    k_reorth_again<<<nvec, FIN_THREADS, 0, st>>>(S, part, RED_BLOCKS);
                    KRY_CHECK_LAUNCH();
                    reorth_dots(Wn, j);
                }
                k_reorth_coef<<<nvec, FIN_THREADS, 0, st>>>(S, dpart, RED_BLOCKS, nsteps, j,
                                                            hstore ? 1.0 / (double)p : 0.0);
                KRY_CHECK_LAUNCH();
                reorth_apply(Wn, j);
            }
        }
        k_lanczos_beta<<<nvec, FIN_THREADS, 0, st>>>(S, part, RED_BLOCKS, nvec, nsteps, j);
        KRY_CHECK_LAUNCH();
        if (hstore) store_half(j + 1);
    };
    step(0);
    if (nsteps > 1)
        run_captured(ctx, [&]() {
            for (int j = 1; j < nsteps; ++j) step(j);
        });
    k_quadrature<<<(nvec + 63) / 64, 64, 0, ctx->stream>>>(S, nvec, nsteps, (double)p, res, e->cov.tau2,
                                                         e->ntheta > 1 ? e->tau2_dev : nullptr, vpt);
    KRY_CHECK_LAUNCH();
    KRY_CUDA(cudaMemcpyAsync(per_vec, res, nvec * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    KRY_CUDA(cudaStreamSynchronize(ctx->stream));
}

void logdet(kry_ctx* ctx, const kry_embed* e, int nprobe, int nsteps, uint64_t seed, bool reorth,
            double* per_probe) {
    KRY_REQUIRE(nsteps >= 1 && nsteps <= KRY_MAX_STEPS, KRY_EINVAL, "nsteps must be in [1, 256]");
    KRY_REQUIRE(nprobe >= 1, KRY_EINVAL, "nprobe must be >= 1");
    if (e->prec == KRY_F64)
        lanczos_logdet<double>(ctx, e, nprobe, nprobe, nsteps, seed, per_probe, 0, reorth);
    else
        lanczos_logdet<float>(ctx, e, nprobe, nprobe, nsteps, seed, per_probe, 0, reorth);
}

// Batched form: ntheta settings of a batched embedding x nprobe probes each
// (nprobe even), per_vec[ntheta * nprobe].
void logdet_batched(kry_ctx* ctx, const kry_embed* e, int nprobe, int nsteps, uint64_t seed, bool reorth,
                    double* per_vec) {
    KRY_REQUIRE(nsteps >= 1 && nsteps <= KRY_MAX_STEPS, KRY_EINVAL, "nsteps must be in [1, 256]");
    KRY_REQUIRE(nprobe >= 2 && nprobe % 2 == 0, KRY_EINVAL, "batched log-det needs an even probe count");
    const int nvec = e->ntheta * nprobe;
    const int vpt = e->ntheta > 1 ? nprobe : 0;
    if (e->prec == KRY_F64)
        lanczos_logdet<double>(ctx, e, nvec, nprobe, nsteps, seed, per_vec, vpt, reorth);
    else
        lanczos_logdet<float>(ctx, e, nvec, nprobe, nsteps, seed, per_vec, vpt, reorth);
}

// ------------------------------------------------------------------ CG

struct CgState {
    double* rr;      // [nrhs] r^T r
    double* alpha;   // [nrhs]
    double* beta;    // [nrhs]
    double* thr2;    // [nrhs] convergence threshold on r^T r
    int* done;       // [nrhs]
    int* iters;      // [nrhs]
    int* ndone;      // [1]
};

// x = 0, r = b (converted), p = r; partial ||r||^2.
template <typename T>
__global__ void k_cg_start(const double* __restrict__ B, int64_t ldb, T* __restrict__ X, T* __restrict__ R,
                           T* __restrict__ P, int64_t p, double* __restrict__ part) {
    const int k = blockIdx.y;
    const int64_t off = (int64_t)k * p;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const T b = (T)B[(int64_t)k * ldb + i];
        X[off + i] = (T)0;
        R[off + i] = b;
        P[off + i] = b;
        acc[0] += (double)b * (double)b;
    }
    block_sum_store<1>(acc, part + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

__global__ void k_cg_init_scalars(CgState S, const double* __restrict__ part, int nblk, int nrhs,
                                  const double* __restrict__ tol) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)k * nblk + b];
    S.rr[k] = s;
    S.thr2[k] = tol[k] * tol[k] * s;
    S.done[k] = (s == 0.0 || s <= S.thr2[k]) ? 1 : 0;
    S.iters[k] = 0;
    S.alpha[k] = 0.0;
    S.beta[k] = 0.0;
    if (k == 0) *S.ndone = 0;
}

__global__ void k_cg_alpha(CgState S, const double* __restrict__ part, int nblk, int nrhs) {
    const int k = blockIdx.x;   // one block per right-hand side
    const double pq = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x == 0) S.alpha[k] = (S.done[k] || pq == 0.0) ? 0.0 : S.rr[k] / pq;
    if (k == 0 && threadIdx.x == 0) *S.ndone = 0;
}

// x += alpha p, r -= alpha q; partial ||r||^2.
template <typename T>
__global__ void k_cg_update(T* __restrict__ X, T* __restrict__ R, const T* __restrict__ P, const T* __restrict__ Q,
                            int64_t p, CgState S, double* __restrict__ part) {
    const int k = blockIdx.y;
    const int64_t off = (int64_t)k * p;
    const T a = (T)S.alpha[k];
    const bool act = !S.done[k];
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        T r = R[off + i];
        if (act) {
            X[off + i] += a * P[off + i];
            r -= a * Q[off + i];
            R[off + i] = r;
        }
        acc[0] += (double)r * (double)r;
    }
    block_sum_store<1>(acc, part + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

__global__ void k_cg_beta(CgState S, const double* __restrict__ part, int nblk, int nrhs, int maxit) {
    const int k = blockIdx.x;   // one block per right-hand side
    const double s = block_sum(part + (int64_t)k * nblk, nblk);
    if (threadIdx.x != 0) return;
    if (!S.done[k]) {
        S.iters[k] += 1;
        S.beta[k] = s / S.rr[k];
        S.rr[k] = s;
        if (s <= S.thr2[k] || !(s == s) || S.iters[k] >= maxit) {
            S.done[k] = 1;
            S.beta[k] = 0.0;
        }
    } else {
        S.beta[k] = 0.0;
    }
    if (S.done[k]) atomicAdd(S.ndone, 1);
}

template <typename T>
__global__ void k_cg_pupdate(T* __restrict__ P, const T* __restrict__ R, int64_t p, CgState S) {
    const int k = blockIdx.y;
    if (S.done[k]) return;
    const int64_t off = (int64_t)k * p;
    const T b = (T)S.beta[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
        P[off + i] = R[off + i] + b * P[off + i];
}

// Inner CG in precision T on nrhs right-hand sides B (FP64, leading dim ldb),
// tolerances tol[k] relative to ||B_k||.  Solution X (T, leading dim p) in
// ctx->work[6].  Returns the largest iteration count.
template <typename T>
static int cg_inner(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, int nrhs, const double* tol_dev,
                    int maxit, T** X_out, int vpt) {
    const bool dbl = sizeof(T) == 8;
    const int64_t p = ctx->p;
    cudaStream_t st = ctx->stream;
    const size_t vb = (size_t)nrhs * p * sizeof(T);
    ctx->work[6].ensure(vb);
    ctx->work[7].ensure(vb);
    ctx->work[8].ensure(vb);
    ctx->work[9].ensure(vb);
    T* X = ctx->work[6].as<T>();
    T* R = ctx->work[7].as<T>();
    T* P = ctx->work[8].as<T>();
    T* Q = ctx->work[9].as<T>();
    const int nblkC = matvec_num_partials(ctx, e, dbl, nrhs);
    ctx->work[10].ensure((size_t)nrhs * std::max(nblkC, RED_BLOCKS) * sizeof(double));
    double* part = ctx->work[10].as<double>();
    ctx->work[11].ensure((size_t)nrhs * (5 * sizeof(double) + 2 * sizeof(int)) + 64);
    char* sb = ctx->work[11].as<char>();
    CgState S;
    S.rr = reinterpret_cast<double*>(sb);
    S.alpha = S.rr + nrhs;
    S.beta = S.alpha + nrhs;
    S.thr2 = S.beta + nrhs;
    S.done = reinterpret_cast<int*>(S.thr2 + nrhs);
    S.iters = S.done + nrhs;
    S.ndone = S.iters + nrhs;

    dim3 gv(RED_BLOCKS, nrhs);
    const int tb = 128;
    k_cg_start<T><<<gv, 256, 0, st>>>(B, ldb, X, R, P, p, part);
    KRY_CHECK_LAUNCH();
    k_cg_init_scalars<<<(nrhs + tb - 1) / tb, tb, 0, st>>>(S, part, RED_BLOCKS, nrhs, tol_dev);
    KRY_CHECK_LAUNCH();
    int* hdone = reinterpret_cast<int*>(ctx->host_pinned);
    int it = 0;
    const int poll = 8;
    for (; it < maxit; ++it) {
        matvec_ex<T>(ctx, e, P, p, nullptr, Q, p, nrhs, part, nblkC, vpt);
        k_cg_alpha<<<nrhs, FIN_THREADS, 0, st>>>(S, part, nblkC, nrhs);
        KRY_CHECK_LAUNCH();
        k_cg_update<T><<<gv, 256, 0, st>>>(X, R, P, Q, p, S, part);
        KRY_CHECK_LAUNCH();
        k_cg_beta<<<nrhs, FIN_THREADS, 0, st>>>(S, part, RED_BLOCKS, nrhs, maxit);
        KRY_CHECK_LAUNCH();
        k_cg_pupdate<T><<<gv, 256, 0, st>>>(P, R, p, S);
        KRY_CHECK_LAUNCH();
        if ((it + 1) % poll == 0) {
            KRY_CUDA(cudaMemcpyAsync(hdone, S.ndone, sizeof(int), cudaMemcpyDeviceToHost, st));
            KRY_CUDA(cudaStreamSynchronize(st));
            if (*hdone >= nrhs) {
                ++it;
                break;
            }
        }
    }
    std::vector<int> its(nrhs);
    KRY_CUDA(cudaMemcpyAsync(hdone, S.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaStreamSynchronize(st));
    int mx = 0;
    for (int k = 0; k < nrhs; ++k) mx = std::max(mx, hdone[k]);
    *X_out = X;
    return mx;
}

__global__ void k_residual(const double* __restrict__ B, int64_t ldb, const double* __restrict__ KX,
                           double* __restrict__ R, int64_t p, double* __restrict__ part) {
    const int k = blockIdx.y;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const double b = B[(int64_t)k * ldb + i];
        const double r = b - KX[(int64_t)k * p + i];
        R[(int64_t)k * p + i] = r;
        acc[0] += r * r;
        acc[1] += b * b;
    }
    block_sum_store<2>(acc, part + ((int64_t)k * gridDim.x + blockIdx.x) * 2, 1);
}

__global__ void k_norms_final(const double* __restrict__ part, int nblk, int nrhs, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    double a = 0.0, b = 0.0;
    for (int j = 0; j < nblk; ++j) {
        a += part[((int64_t)k * nblk + j) * 2];
        b += part[((int64_t)k * nblk + j) * 2 + 1];
    }
    out[2 * k] = sqrt(a);
    out[2 * k + 1] = sqrt(b);
}

__global__ void k_set(double* x, int64_t n, double v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// FP64 true residual R = B - K X; returns per-column (||R||, ||B||) on the host.
static void true_residual(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, const double* X,
                          int64_t ldx, int nrhs, double* R, double* KX, std::vector<double>& nrm, int vpt,
                          const int* skip) {
    const int64_t p = ctx->p;
    cudaStream_t st = ctx->stream;
    // KX = K X (FP64 matvec); X has leading dimension ldx.  Columns flagged in
    // skip (pairs of them) are not transformed: their residual norms are stale.
    matvec_ex<double>(ctx, e, X, ldx, nullptr, KX, p, nrhs, nullptr, 0, vpt, skip);
    ctx->red.ensure((size_t)nrhs * RED_BLOCKS * 2 * sizeof(double) + (size_t)nrhs * 2 * sizeof(double));
    double* part = ctx->red.as<double>();
    double* fin = part + (size_t)nrhs * RED_BLOCKS * 2;
    dim3 gv(RED_BLOCKS, nrhs);
    k_residual<<<gv, 256, 0, st>>>(B, ldb, KX, R, p, part);
    KRY_CHECK_LAUNCH();
    k_norms_final<<<(nrhs + 127) / 128, 128, 0, st>>>(part, RED_BLOCKS, nrhs, fin);
    KRY_CHECK_LAUNCH();
    nrm.resize(2 * nrhs);
    KRY_CUDA(cudaMemcpyAsync(nrm.data(), fin, 2 * nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ reliable-update mixed-precision CG
//
// FP32 CG (FP32 matvec, FP64 scalars) whose solution accumulates in FP64 and
// whose recursive FP32 residual is replaced by the true residual b - K x,
// computed with the FP64 matvec, whenever it has fallen 10x since the last
// replacement or reached the target (the "reliable updates" of van der Vorst
// & Ye, "Residual replacement strategies for Krylov subspace iterative
// methods", SIAM J. Sci. Comput. 2000).  The search direction is kept across
// replacements, so the Krylov progress of FP64 CG is retained while every
// matvec of the iteration runs in FP32.  Convergence is declared only on a
// true FP64 residual.

// Each iteration is the plain CG recurrence on five launches, none of which
// starts with a reduction:
//   q = K p                      (FFT matvec; pass C forms the partials of p^T q)
//   alpha = gamma / p^T q        (k_rcg_alpha: one block per column, fixed-order sum)
//   x += alpha p, r -= alpha q   (k_rcg_update: streaming, forms the partials of r^T r)
//   beta = gamma' / gamma        (k_rcg_beta: one block per column; counts the iteration
//                                 and asks for a residual replacement)
//   p = r + beta p               (k_rcg_pupdate: streaming)
// K p is computed afresh by every matvec, so no auxiliary recurrence can
// drift in FP32 (single-reduction rearrangements carry K p by a recurrence and
// broke down on the ill-conditioned grids here).
//
// With a preconditioner (an embedding `pre` whose matvec applies M^-1 = A (S +
// tau2 I)^-1 A^T, S the circulant embedding of sigma2 Sigma on the matvec's
// torus: the inverse of the torus covariance, restricted to the observed
// cells), the same launches run preconditioned CG: after the update, z = M^-1 r
// by the FFT passes (pass C forms the partials of r^T z), gamma = r^T z,
// beta = gamma' / gamma, p = z + beta p; convergence is still judged on r^T r.
// M^-1 is symmetric positive definite (a principal block of an SPD matrix).
// It approximates K^-1 well where most of the grid is observed and the gaps
// are clustered, and poorly under scattered missing cells.
struct RcgState {
    double* gam;      // [nrhs] gamma = r^T z (r^T r without a preconditioner)
    double* rr;       // [nrhs] r^T r of the current residual
    double* alpha;    // [nrhs]
    double* beta;     // [nrhs]
    double* rr_ref;   // [nrhs] r^T r at the last replacement
    double* thr2;     // [nrhs] (rtol ||b||)^2
    int* want;        // [nrhs] 1: the last iteration asks for a replacement
    int* done;        // [nrhs]
    int* iters;       // [nrhs]
    int* ndone;       // [1]
};

// Blocks per right-hand side of the CG vector kernels: 304 (two per SM) for a
// few right-hand sides, fewer for many, so that a batch keeps about 1216
// blocks.
static int cg_blocks(int nrhs) { return std::max(8, std::min(304, 1216 / std::max(1, nrhs))); }

// X = 0 (a double-float pair Xh + Xl), R = P = (float) B; partials of ||B||^2
// (FP64) per column, one per block.
__global__ void k_rcg_start(const double* __restrict__ B, int64_t ldb, float* __restrict__ Xh, float* __restrict__ Xl,
                            float* __restrict__ R, float* __restrict__ P, int64_t p, double* __restrict__ part_rr) {
    const int k = blockIdx.y;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const double b = B[(int64_t)k * ldb + i];
        const int64_t o = (int64_t)k * p + i;
        Xh[o] = 0.f;
        Xl[o] = 0.f;
        R[o] = (float)b;
        P[o] = (float)b;
        acc[0] += b * b;
    }
    block_sum_store<1>(acc, part_rr + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

// rr = ||B||^2 from the start's partials; gamma = r^T z from the
// preconditioner matvec's partials (part_rz, nrz per column) or = rr.
__global__ void k_rcg_init_scalars(RcgState S, const double* __restrict__ part_rr, int nblk,
                                   const double* __restrict__ part_rz, int nrz, int nrhs,
                                   const double* __restrict__ tol) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrhs) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part_rr[(int64_t)k * nblk + b];
        double g = s;
        if (part_rz) {
            g = 0.0;
            for (int b = 0; b < nrz; ++b) g += part_rz[(int64_t)k * nrz + b];
        }
        S.gam[k] = g;
        S.rr[k] = s;
        S.rr_ref[k] = s;
        S.alpha[k] = 0.0;
        S.beta[k] = 0.0;
        S.thr2[k] = tol[k] * tol[k] * s;
        S.want[k] = 0;
        S.done[k] = (s == 0.0 || !(g > 0.0)) ? 1 : 0;
        S.iters[k] = 0;
    }
}

// alpha = gamma / p^T q from the matvec's partials (fixed order; 0 if p^T q is
// not positive).
__global__ void k_rcg_alpha(RcgState S, const double* __restrict__ part_pq, int nblkC) {
    pdl_wait();
    pdl_launch_dependents();
    const int k = blockIdx.x;
    if (S.done[k]) return;
    const double d = block_sum(part_pq + (int64_t)k * nblkC, nblkC);
    if (threadIdx.x == 0) S.alpha[k] = (d > 0.0) ? S.gam[k] / d : 0.0;
}

// X += alpha P in double-float (Xh + Xl, FP32 instructions only), R -= alpha Q
// (FP32); partials of ||R||^2 in double-float.  VW elements per 16-byte access
// (the internal vectors are 16-byte aligned when p % 4 == 0).
template <int VW>
__global__ void k_rcg_update(float* __restrict__ Xh, float* __restrict__ Xl, float* __restrict__ R,
                             const float* __restrict__ P, const float* __restrict__ Q, int64_t p, RcgState S,
                             double* __restrict__ part_rr) {
    pdl_wait();
    pdl_launch_dependents();
    const int k = blockIdx.y;
    if (S.done[k]) return;   // finished columns keep x and r
    const double a = S.alpha[k];
    const float af = (float)a;
    float ahi, alo;
    df_split(a, ahi, alo);
    const int64_t off = (int64_t)k * p;
    const int64_t nv = p / VW;
    DFAcc nrm;
    for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv; xv += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = off + xv * VW;
        float r[VW], pv[VW], qv[VW], xh[VW], xl[VW];
        load_vec<float, VW>(R + o, r);
        load_vec<float, VW>(P + o, pv);
        load_vec<float, VW>(Q + o, qv);
        load_vec<float, VW>(Xh + o, xh);
        load_vec<float, VW>(Xl + o, xl);
#pragma unroll
        for (int e = 0; e < VW; ++e) {
            df_axpy(xh[e], xl[e], ahi, alo, pv[e]);
            r[e] -= af * qv[e];
            nrm.add_prod(r[e], r[e]);
        }
        store_vec<float, VW>(Xh + o, xh);
        store_vec<float, VW>(Xl + o, xl);
        store_vec<float, VW>(R + o, r);
    }
    double acc[1] = {nrm.value()};
    block_sum_store<1>(acc, part_rr + (int64_t)k * gridDim.x + blockIdx.x, 0);
}

// rr' = r^T r from the update's partials and gamma' = r^T z from part_rz (nrz
// per column; NULL without a preconditioner: gamma' = rr'), both in a fixed
// order; beta = gamma' / gamma.  Counts the iteration and asks for a
// replacement when rr' has fallen 100x since the last one, reached the
// target, is not finite, or the budget is spent.
__global__ void k_rcg_beta(RcgState S, const double* __restrict__ part_rr, int nbc, const double* __restrict__ part_rz,
                           int nrz, int maxit) {
    pdl_wait();
    pdl_launch_dependents();
    const int k = blockIdx.x;
    if (S.done[k]) return;
    const double rr = block_sum(part_rr + (int64_t)k * nbc, nbc);
    double g = rr;
    if (part_rz) {
        __syncthreads();   // block_sum's shared slots are reused
        g = block_sum(part_rz + (int64_t)k * nrz, nrz);
    }
    if (threadIdx.x == 0) {
        const double g0 = S.gam[k];
        S.beta[k] = (g0 > 0.0) ? g / g0 : 0.0;
        S.gam[k] = g;
        S.rr[k] = rr;
        const int it = S.iters[k] + 1;
        S.iters[k] = it;
        S.want[k] = (rr <= S.thr2[k] || rr <= 1e-2 * S.rr_ref[k] || !(rr == rr) || !(g == g) || it >= maxit) ? 1 : 0;
    }
}

// P = Z + beta P (FP32); Z = R without a preconditioner.
template <int VW>
__global__ void k_rcg_pupdate(float* __restrict__ P, const float* __restrict__ Z, int64_t p, RcgState S) {
    pdl_wait();
    pdl_launch_dependents();
    const int k = blockIdx.y;
    if (S.done[k]) return;
    const float b = (float)S.beta[k];
    float* Pk = P + (int64_t)k * p;
    const float* Zk = Z + (int64_t)k * p;
    const int64_t nv = p / VW;
    for (int64_t xv = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xv < nv; xv += (int64_t)gridDim.x * blockDim.x) {
        float z[VW], pv[VW];
        load_vec<float, VW>(Zk + xv * VW, z);
        load_vec<float, VW>(Pk + xv * VW, pv);
#pragma unroll
        for (int e = 0; e < VW; ++e) pv[e] = z[e] + b * pv[e];
        store_vec<float, VW>(Pk + xv * VW, pv);
    }
}

// X = Xh + Xl in FP64 (the caller's layout, leading dimension ldx).
__global__ void k_df_to_f64(const float* __restrict__ Xh, const float* __restrict__ Xl, int64_t p,
                            double* __restrict__ X, int64_t ldx) {
    const int k = blockIdx.y;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
        X[(int64_t)k * ldx + i] = (double)Xh[(int64_t)k * p + i] + (double)Xl[(int64_t)k * p + i];
}

// Residual replacement of the running columns of the round: R = (float) R64,
// rr = rr_ref = ||R64||^2 and, without a preconditioner, gamma = rr (P is
// kept); done when ||R64|| <= rtol ||B|| or the iteration budget is spent (a
// non-finite residual also ends the column; the caller reports it).
__global__ void k_rcg_replace(const double* __restrict__ R64, float* __restrict__ R, int64_t p,
                              const double* __restrict__ norms, RcgState S, int maxit, int precond,
                              const int* __restrict__ sel) {
    const int k = blockIdx.y;
    if (S.done[k] || sel[k]) return;   // only the columns of the round (the others' norms are stale)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
        R[(int64_t)k * p + i] = (float)R64[(int64_t)k * p + i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // (want is cleared by k_count_done, after every block)
        const double rn = norms[2 * k];
        if (!precond) S.gam[k] = rn * rn;
        S.rr[k] = rn * rn;
        S.rr_ref[k] = rn * rn;
        if (rn * rn <= S.thr2[k] || S.iters[k] >= maxit || !(rn == rn)) S.done[k] = 1;
    }
}

// gamma = r^T z after a replacement (preconditioned runs): the fixed-order sum
// of the preconditioner matvec's partials.
__global__ void k_rcg_regamma(RcgState S, const double* __restrict__ part_rz, int nrz, const int* __restrict__ sel) {
    const int k = blockIdx.x;
    if (S.done[k] || sel[k]) return;
    const double g = block_sum(part_rz + (int64_t)k * nrz, nrz);
    if (threadIdx.x == 0) S.gam[k] = g;
}

// Ends a replacement round: counts the finished columns and clears the requests.
__global__ void k_count_done(RcgState S, int nrhs) {
    int d = 0;
    for (int k = 0; k < nrhs; ++k) {
        d += S.done[k];
        S.want[k] = 0;
    }
    *S.ndone = d;
}

static void true_residual(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, const double* X,
                          int64_t ldx, int nrhs, double* R, double* KX, std::vector<double>& nrm, int vpt,
                          const int* skip = nullptr);

// Skip flags of a replacement round: with `all`, no column is skipped (every
// running column is replaced, and the FP64 residual covers the finished ones
// too); otherwise the columns that are done or do not ask for a replacement.
__global__ void k_rcg_select(RcgState S, int nrhs, int* __restrict__ skip, int all) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nrhs) skip[k] = (!all && (S.done[k] || !S.want[k])) ? 1 : 0;
}

// Returns the largest per-column iteration count.  pre: preconditioner
// embedding (NULL: plain CG).
static int cg_reliable(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, double* X, int64_t ldx,
                       int nrhs, double rtol, int maxit, std::vector<double>& nrm, bool* fresh, int vpt,
                       const kry_embed* pre) {
    const int64_t p = ctx->p;
    cudaStream_t st = ctx->stream;
    const size_t vb = (size_t)nrhs * p * sizeof(float);
    ctx->work[7].ensure(vb);
    ctx->work[8].ensure(vb);
    ctx->work[9].ensure(vb);
    float* R = ctx->work[7].as<float>();
    float* P = ctx->work[8].as<float>();
    float* Q = ctx->work[9].as<float>();
    float* Z = R;
    if (pre) {
        ctx->work[3].ensure(vb);
        Z = ctx->work[3].as<float>();
    }
    const int nblkC = matvec_num_partials(ctx, e, false, nrhs);
    const int nbc = cg_blocks(nrhs);
    ctx->work[10].ensure((size_t)nrhs * (2 * nblkC + nbc) * sizeof(double));
    double* part_pq = ctx->work[10].as<double>();        // matvec partials (p^T K p)
    double* part_rr = part_pq + (size_t)nrhs * nblkC;     // start / update partials (r^T r)
    double* part_rz = pre ? part_rr + (size_t)nrhs * nbc : nullptr;   // preconditioner partials (r^T z)
    ctx->work[11].ensure((size_t)nrhs * (6 * sizeof(double) + 4 * sizeof(int)) + 64);
    char* sb = ctx->work[11].as<char>();
    RcgState S;
    S.gam = reinterpret_cast<double*>(sb);
    S.rr = S.gam + nrhs;
    S.alpha = S.rr + nrhs;
    S.beta = S.alpha + nrhs;
    S.rr_ref = S.beta + nrhs;
    S.thr2 = S.rr_ref + nrhs;
    S.want = reinterpret_cast<int*>(S.thr2 + nrhs);
    S.done = S.want + nrhs;
    S.iters = S.done + nrhs;
    S.ndone = S.iters + nrhs;
    int* sel = S.ndone + 1;   // skip flags of a replacement round
    ctx->tolbuf.ensure(nrhs * sizeof(double));
    std::vector<double> tol_h(nrhs, rtol);
    KRY_CUDA(cudaMemcpyAsync(ctx->tolbuf.p, tol_h.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    ctx->work[4].ensure((size_t)nrhs * p * sizeof(double));
    double* R64 = ctx->work[4].as<double>();
    ctx->kxbuf.ensure((size_t)nrhs * p * sizeof(double));
    ctx->work[12].ensure(2 * vb);
    float* Xh = ctx->work[12].as<float>();   // the solution as a double-float pair
    float* Xl = Xh + (size_t)nrhs * p;

    dim3 gv(RED_BLOCKS, nrhs);
    dim3 gc(nbc, nrhs);
    const int tbeta = std::max(32, ((nrhs + 31) / 32) * 32);
    const bool vec = p % 4 == 0;   // 16-byte accesses: every column start is 16-byte aligned
    auto to_f64 = [&]() {
        k_df_to_f64<<<gv, 256, 0, st>>>(Xh, Xl, p, X, ldx);
        KRY_CHECK_LAUNCH();
    };
    k_rcg_start<<<gc, 256, 0, st>>>(B, ldb, Xh, Xl, R, P, p, part_rr);
    KRY_CHECK_LAUNCH();
    if (pre) matvec_ex<float>(ctx, pre, R, p, nullptr, Z, p, nrhs, part_rz, nblkC, vpt, nullptr);   // z = M^-1 r
    k_rcg_init_scalars<<<1, tbeta, 0, st>>>(S, part_rr, nbc, part_rz, nblkC, nrhs, ctx->tolbuf.as<double>());
    KRY_CHECK_LAUNCH();
    if (pre) {   // p = z (beta = 0)
        launch_pdl(vec ? k_rcg_pupdate<4> : k_rcg_pupdate<1>, gc, dim3(256), 0, st, P, (const float*)Z, p, S);
    }
    int* hflag = reinterpret_cast<int*>(ctx->host_pinned);
    const int poll = 8;
    nrm.assign(2 * nrhs, 0.0);
    *fresh = false;
    // one CG iteration on ctx->stream (the capture stream while capturing)
    auto iterate = [&]() {
        cudaStream_t s2 = ctx->stream;
        // kernels launched back to back with programmatic dependent launch: each
        // waits for its predecessor's completion before touching its outputs;
        // columns that have converged are not transformed (pairs of finished
        // columns skip every pass)
        matvec_ex<float>(ctx, e, P, p, nullptr, Q, p, nrhs, part_pq, nblkC, vpt, S.done);
        launch_pdl(k_rcg_alpha, dim3(nrhs), dim3(FIN_THREADS), 0, s2, S, part_pq, nblkC);
        launch_pdl(vec ? k_rcg_update<4> : k_rcg_update<1>, gc, dim3(256), 0, s2, Xh, Xl, R, P, Q, p, S, part_rr);
        if (pre) matvec_ex<float>(ctx, pre, R, p, nullptr, Z, p, nrhs, part_rz, nblkC, vpt, S.done);
        launch_pdl(k_rcg_beta, dim3(nrhs), dim3(FIN_THREADS), 0, s2, S, part_rr, nbc, (const double*)part_rz, nblkC,
                   maxit);
        launch_pdl(vec ? k_rcg_pupdate<4> : k_rcg_pupdate<1>, gc, dim3(256), 0, s2, P, (const float*)Z, p, S);
    };
    // Iterations run in blocks of `poll`.  The first block runs directly (it
    // sizes every buffer); later blocks replay one captured graph.
    Replay block(ctx);
    for (int it0 = 0; it0 < maxit + poll; it0 += poll) {
        if (it0 == 0 || !ctx->use_graphs) {
            for (int i = 0; i < poll; ++i) iterate();
        } else {
            if (!block.exec)
                block.capture([&]() {
                    for (int i = 0; i < poll; ++i) iterate();
                });
            block.launch();
        }
        KRY_CUDA(cudaMemcpyAsync(hflag, S.want, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
        KRY_CUDA(cudaStreamSynchronize(st));
        if (block.exec) block.harvest();
        int nwant = 0;
        for (int k = 0; k < nrhs; ++k) nwant += hflag[k] != 0;
        if (nwant > 0) {
            // Residual replacement.  A few right-hand sides (which converge
            // together) are all replaced in one round; in larger batches only
            // the columns that ask for it, and the FP64 matvec transforms only
            // their pairs.
            const int all = nrhs <= 8 ? 1 : 0;
            k_rcg_select<<<1, tbeta, 0, st>>>(S, nrhs, sel, all);
            KRY_CHECK_LAUNCH();
            to_f64();
            true_residual(ctx, e, B, ldb, X, ldx, nrhs, R64, ctx->kxbuf.as<double>(), nrm, vpt, sel);
            double* dn = ctx->red.as<double>() + (size_t)nrhs * RED_BLOCKS * 2;   // device norms
            k_rcg_replace<<<gc, 256, 0, st>>>(R64, R, p, dn, S, maxit, pre ? 1 : 0, sel);
            KRY_CHECK_LAUNCH();
            if (pre) {   // z = M^-1 r and gamma = r^T z for the replaced r
                matvec_ex<float>(ctx, pre, R, p, nullptr, Z, p, nrhs, part_rz, nblkC, vpt, sel);
                k_rcg_regamma<<<nrhs, FIN_THREADS, 0, st>>>(S, part_rz, nblkC, sel);
                KRY_CHECK_LAUNCH();
            }
            k_count_done<<<1, 1, 0, st>>>(S, nrhs);
            KRY_CHECK_LAUNCH();
            KRY_CUDA(cudaMemcpyAsync(hflag, S.ndone, sizeof(int), cudaMemcpyDeviceToHost, st));
            KRY_CUDA(cudaStreamSynchronize(st));
            if (*hflag >= nrhs) {
                // the last residuals are every column's only if every column took part
                *fresh = all || nwant == nrhs;
                break;
            }
        }
    }
    to_f64();   // X, after the loop or its last replacement round (idempotent)
    std::vector<int> its(nrhs);
    KRY_CUDA(cudaMemcpyAsync(its.data(), S.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaStreamSynchronize(st));
    int mx = 0;
    for (int k = 0; k < nrhs; ++k) mx = std::max(mx, its[k]);
    return mx;
}

SolveInfo solve(kry_ctx* ctx, const kry_embed* e, const double* B, int64_t ldb, double* X, int64_t ldx, int nrhs,
                double rtol, int maxit, int vpt = 0, const kry_embed* pre = nullptr) {
    SolveInfo info;
    const int64_t p = ctx->p;
    cudaStream_t st = ctx->stream;
    KRY_REQUIRE(nrhs >= 1, KRY_EINVAL, "nrhs must be >= 1");
    KRY_REQUIRE(rtol > 0 && maxit >= 1, KRY_EINVAL, "rtol must be > 0 and maxit >= 1");
    ctx->kxbuf.ensure((size_t)nrhs * p * sizeof(double));
    ctx->work[4].ensure((size_t)nrhs * p * sizeof(double));
    double* R = ctx->work[4].as<double>();
    std::vector<double> nrm;
    bool fresh = false;
    if (e->prec == KRY_F64) {
        // plain FP64 CG
        ctx->tolbuf.ensure(nrhs * sizeof(double));
        std::vector<double> tol_h(nrhs, rtol);
        KRY_CUDA(cudaMemcpyAsync(ctx->tolbuf.p, tol_h.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
        double* Xd;
        info.iters = cg_inner<double>(ctx, e, B, ldb, nrhs, ctx->tolbuf.as<double>(), maxit, &Xd, vpt);
        KRY_CUDA(cudaMemcpy2DAsync(X, ldx * sizeof(double), Xd, p * sizeof(double), p * sizeof(double), nrhs,
                                   cudaMemcpyDeviceToDevice, st));
    } else {
        // FP32 CG with FP64 solution and residual replacement
        info.iters = cg_reliable(ctx, e, B, ldb, X, ldx, nrhs, rtol, maxit, nrm, &fresh, vpt, pre);
    }
    // the reported residual is always the true FP64 residual of the returned X
    if (!fresh) true_residual(ctx, e, B, ldb, X, ldx, nrhs, R, ctx->kxbuf.as<double>(), nrm, vpt);
    info.relres = 0.0;
    for (int k = 0; k < nrhs; ++k) {
        const double bn = nrm[2 * k + 1];
        const double rk = bn > 0 ? nrm[2 * k] / bn : 0.0;
        if (!(rk == rk)) {   // a non-finite residual is reported, not dropped by max
            info.relres = rk;
            break;
        }
        info.relres = std::max(info.relres, rk);
    }
    info.converged = info.relres <= rtol * (1.0 + 1e-9);
    return info;
}

// ------------------------------------------------------------------ GLS and the log-likelihood

// G[a][b] = V_a^T Z_b for the (ncov+1) columns V = [y, X] and Z = K^-1 V.
__global__ void k_gram(const double* __restrict__ V, int64_t ldv, const double* __restrict__ Z, int64_t ldz,
                       int64_t p, int nc, double* __restrict__ part) {
    const int a = blockIdx.y / nc, b = blockIdx.y % nc;
    double acc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += V[(int64_t)a * ldv + i] * Z[(int64_t)b * ldz + i];
    block_sum_store<1>(acc, part + (int64_t)blockIdx.y * gridDim.x + blockIdx.x, 0);
}

// beta = (X^T K^-1 X)^-1 X^T K^-1 y by Cholesky of the ncov x ncov matrix;
// quad = y^T K^-1 y - beta^T X^T K^-1 y; loglik = -1/2 (logdet + quad + p log 2 pi).
__global__ void k_gls(const double* __restrict__ part, int nblk, int ncov, int64_t p, double logdet,
                      double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nc = ncov + 1;
    double G[KRY_MAX_COV + 1][KRY_MAX_COV + 1];
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nc; ++b) {
            double s = 0.0;
            for (int j = 0; j < nblk; ++j) s += part[(int64_t)(a * nc + b) * nblk + j];
            G[a][b] = s;
        }
    // symmetrise (V^T K^-1 V is symmetric in exact arithmetic)
    double A[KRY_MAX_COV][KRY_MAX_COV], g[KRY_MAX_COV], L[KRY_MAX_COV][KRY_MAX_COV];
    for (int a = 0; a < ncov; ++a) {
        g[a] = 0.5 * (G[a + 1][0] + G[0][a + 1]);
        for (int b = 0; b < ncov; ++b) A[a][b] = 0.5 * (G[a + 1][b + 1] + G[b + 1][a + 1]);
    }
    int ok = 1;
    for (int j = 0; j < ncov; ++j) {
        double s = A[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0)) {
            ok = 0;
            s = 1e-300;
        }
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < ncov; ++i) {
            double t = A[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    double w[KRY_MAX_COV], beta[KRY_MAX_COV];
    for (int i = 0; i < ncov; ++i) {
        double t = g[i];
        for (int k = 0; k < i; ++k) t -= L[i][k] * w[k];
        w[i] = t / L[i][i];
    }
    for (int i = ncov - 1; i >= 0; --i) {
        double t = w[i];
        for (int k = i + 1; k < ncov; ++k) t -= L[k][i] * beta[k];
        beta[i] = t / L[i][i];
    }
    double quad = G[0][0];
    for (int i = 0; i < ncov; ++i) quad -= beta[i] * g[i];
    const double ll = -0.5 * (logdet + quad + (double)p * 1.8378770664093454836);
    out[0] = ll;
    out[1] = quad;
    out[2] = ok ? 0.0 : 1.0;
    for (int i = 0; i < ncov; ++i) out[3 + i] = beta[i];
}

// V = [y, X] (p x (ncov+1), ld p) and Z = K^-1 V already solved.
GlsResult gls(kry_ctx* ctx, const double* V, const double* Z, int ncov, double logdet) {
    const int64_t p = ctx->p;
    const int nc = ncov + 1;
    cudaStream_t st = ctx->stream;
    ctx->red.ensure((size_t)nc * nc * RED_BLOCKS * sizeof(double) + 64 * sizeof(double));
    double* part = ctx->red.as<double>();
    double* out = part + (size_t)nc * nc * RED_BLOCKS;
    dim3 g(RED_BLOCKS, nc * nc);
    k_gram<<<g, 256, 0, st>>>(V, p, Z, p, p, nc, part);
    KRY_CHECK_LAUNCH();
    k_gls<<<1, 32, 0, st>>>(part, RED_BLOCKS, ncov, p, logdet, out);
    KRY_CHECK_LAUNCH();
    KRY_CUDA(cudaMemcpyAsync(ctx->host_pinned, out, (3 + ncov) * sizeof(double), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaStreamSynchronize(st));
    GlsResult r;
    r.loglik = ctx->host_pinned[0];
    r.quad = ctx->host_pinned[1];
    r.ok = ctx->host_pinned[2] == 0.0;
    for (int i = 0; i < ncov; ++i) r.beta[i] = ctx->host_pinned[3 + i];
    return r;
}

// ------------------------------------------------------------------ kriging helpers

// w = Z[:,0] - Z[:,1:] beta  (K^-1 (y - X beta) without another solve).
__global__ void k_resid_weights(const double* __restrict__ Z, int64_t p, int ncov, const double* __restrict__ beta,
                                double* __restrict__ w) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        double v = Z[i];
        for (int c = 0; c < ncov; ++c) v -= Z[(int64_t)(c + 1) * p + i] * beta[c];
        w[i] = v;
    }
}

// ------------------------------------------------------------------ parametric bootstrap (Sec. 3.5)

__global__ void k_boot_rhs(const double* __restrict__ G, int64_t N, const int* __restrict__ cellidx, int64_t p,
                           const double* __restrict__ eps, double tau, double* __restrict__ R) {
    const int b = blockIdx.y;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p; q += (int64_t)gridDim.x * blockDim.x)
        R[(int64_t)b * p + q] = G[(int64_t)b * N + cellidx[q]] + tau * eps[(int64_t)b * p + q];
}

void boot_rhs(kry_ctx* ctx, const double* G, int64_t N, const double* eps, double tau, double* R, int nrep) {
    const int64_t p = ctx->p;
    dim3 g((unsigned)std::min<int64_t>((p + 255) / 256, 1024), nrep);
    k_boot_rhs<<<g, 256, 0, ctx->stream>>>(G, N, ctx->cellidx.as<int>(), p, eps, tau, R);
    KRY_CHECK_LAUNCH();
}

__global__ void k_boot_mse(const double* __restrict__ G, const double* __restrict__ H, int64_t N, int nrep,
                           const int64_t* __restrict__ cells, int64_t ncell, double* __restrict__ var,
                           int* __restrict__ bad) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = cells[t];
        if (cell < 0 || cell >= N) {
            var[t] = __longlong_as_double(0x7ff8000000000000ll);
            *bad = 1;
            continue;
        }
        double s = 0.0;
        for (int b = 0; b < nrep; ++b) {
            const double d = G[(int64_t)b * N + cell] - H[(int64_t)b * N + cell];
            s += d * d;
        }
        var[t] = s / nrep;
    }
}

void boot_mse(kry_ctx* ctx, const double* G, const double* H, int64_t N, int nrep, const int64_t* cells,
              int64_t ncell, double* var, int* bad) {
    if (ncell <= 0) return;
    k_boot_mse<<<(unsigned)std::min<int64_t>((ncell + 255) / 256, 4096), 256, 0, ctx->stream>>>(G, H, N, nrep, cells,
                                                                                              ncell, var, bad);
    KRY_CHECK_LAUNCH();
}

// mean[t] = X_t beta + grid[cells[t]]; a cell index outside [0, N) gives NaN
// and raises *bad.
__global__ void k_krige_cells(const double* __restrict__ grid, int64_t N, const int64_t* __restrict__ cells,
                              int64_t ncell, const double* __restrict__ Xc, int ncov, const double* __restrict__ beta,
                              double* __restrict__ mean, int* __restrict__ bad) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = cells[t];
        if (cell < 0 || cell >= N) {
            mean[t] = __longlong_as_double(0x7ff8000000000000ll);
            *bad = 1;
            continue;
        }
        double m = grid[cell];
        for (int c = 0; c < ncov; ++c) m += Xc[(int64_t)c * ncell + t] * beta[c];
        mean[t] = m;
    }
}

struct CovPar {
    double sigma2, inv_range, nu, ca, sa, ratio, dx1, dx2;
};

// mean[s] = X_s beta + sum_o sigma2 rho(site_s - cell_o) w_o  (one block per site).
__global__ void k_krige_sites(const double* __restrict__ sites, int64_t nsite, const double* __restrict__ Xs, int ncov,
                              const double* __restrict__ beta, const double* __restrict__ w,
                              const int* __restrict__ cellidx, int64_t p, int n2, CovPar cp,
                              double* __restrict__ mean) {
    const int64_t s = blockIdx.x;
    if (s >= nsite) return;
    const double x1 = sites[2 * s], x2 = sites[2 * s + 1];
    double acc[1] = {0.0};
    for (int64_t q = threadIdx.x; q < p; q += blockDim.x) {
        const int cell = cellidx[q];
        const int i = cell / n2, j = cell - (cell / n2) * n2;
        const double h1 = x1 - (i + 0.5) * cp.dx1, h2 = x2 - (j + 0.5) * cp.dx2;
        const double r = kry_scaled_dist(h1, h2, cp.ca, cp.sa, cp.ratio, cp.inv_range);
        acc[0] += cp.sigma2 * kry_matern(r, cp.nu) * w[q];
    }
    __shared__ double tot;
    block_sum_store<1>(acc, &tot, 0);
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = tot;
        for (int c = 0; c < ncov; ++c) m += Xs[(int64_t)c * nsite + s] * beta[c];
        mean[s] = m;
    }
}

// Columns of sigma2 Sigma_{obs, t} for a batch of target cells: C[k][q].
// Target cells are clamped into the grid (k_krige_cells flags bad indices).
__global__ void k_cross_cols(const int64_t* __restrict__ cells, int64_t t0, const int* __restrict__ cellidx, int64_t p,
                             int n2, int64_t N, CovPar cp, double* __restrict__ C) {
    const int k = blockIdx.y;
    const int64_t t = min(max(cells[t0 + k], (int64_t)0), N - 1);
    const int ti = (int)(t / n2), tj = (int)(t - (t / n2) * n2);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < p; q += (int64_t)gridDim.x * blockDim.x) {
        const int cell = cellidx[q];
        const int i = cell / n2, j = cell - (cell / n2) * n2;
        const double r = kry_scaled_dist((i - ti) * cp.dx1, (j - tj) * cp.dx2, cp.ca, cp.sa, cp.ratio, cp.inv_range);
        C[(int64_t)k * p + q] = cp.sigma2 * kry_matern(r, cp.nu);
    }
}

// var[t0 + k] = sigma2 - C_k^T S_k.
__global__ void k_var_final(const double* __restrict__ C, const double* __restrict__ Sx, int64_t p, double sigma2,
                            double* __restrict__ var, int64_t t0) {
    const int k = blockIdx.x;
    double acc[1] = {0.0};
    for (int64_t q = threadIdx.x; q < p; q += blockDim.x) acc[0] += C[(int64_t)k * p + q] * Sx[(int64_t)k * p + q];
    __shared__ double tot;
    block_sum_store<1>(acc, &tot, 0);
    __syncthreads();
    if (threadIdx.x == 0) var[t0 + k] = sigma2 - tot;
}

CovPar cov_par(const kry_cov& cov, double dx1, double dx2) {
    CovPar c;
    c.sigma2 = cov.sigma2;
    c.inv_range = 1.0 / cov.range;
    c.nu = cov.nu;
    c.ca = cos(cov.aniso_angle);
    c.sa = sin(cov.aniso_angle);
    c.ratio = cov.aniso_ratio;
    c.dx1 = dx1;
    c.dx2 = dx2;
    return c;
}

void krige_launch_cells(kry_ctx* ctx, const double* grid, const int64_t* cells, int64_t ncell, const double* Xc,
                        int ncov, const double* beta_dev, double* mean, int* bad) {
    if (ncell <= 0) return;
    k_krige_cells<<<(unsigned)std::min<int64_t>((ncell + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        grid, (int64_t)ctx->n1 * ctx->n2, cells, ncell, Xc, ncov, beta_dev, mean, bad);
    KRY_CHECK_LAUNCH();
}

void krige_launch_sites(kry_ctx* ctx, const kry_cov& cov, const double* sites, int64_t nsite, const double* Xs,
                        int ncov, const double* beta_dev, const double* w, double* mean) {
    if (nsite <= 0) return;
    k_krige_sites<<<(unsigned)nsite, 256, 0, ctx->stream>>>(sites, nsite, Xs, ncov, beta_dev, w,
                                                           ctx->cellidx.as<int>(), ctx->p, ctx->n2,
                                                           cov_par(cov, ctx->dx1, ctx->dx2), mean);
    KRY_CHECK_LAUNCH();
}

void resid_weights(kry_ctx* ctx, const double* Z, int ncov, const double* beta_dev, double* w) {
    k_resid_weights<<<(unsigned)std::min<int64_t>((ctx->p + 255) / 256, 4096), 256, 0, ctx->stream>>>(
        Z, ctx->p, ncov, beta_dev, w);
    KRY_CHECK_LAUNCH();
}

// Simple-kriging variances at target cells, nb targets per batch of solves.
bool krige_variances(kry_ctx* ctx, const kry_embed* e, const int64_t* cells, int64_t ncell, double* var,
                     double rtol, int maxit, const kry_embed* pre) {
    const int64_t p = ctx->p;
    cudaStream_t st = ctx->stream;
    const int nb = 32;
    DevBuf& cbuf = ctx->cbuf;
    DevBuf& sbuf = ctx->sbuf;
    cbuf.ensure((size_t)nb * p * sizeof(double));
    sbuf.ensure((size_t)nb * p * sizeof(double));
    bool ok = true;
    const CovPar cp = cov_par(e->cov, ctx->dx1, ctx->dx2);
    for (int64_t t0 = 0; t0 < ncell; t0 += nb) {
        const int k = (int)std::min<int64_t>(nb, ncell - t0);
        dim3 g((unsigned)std::min<int64_t>((p + 255) / 256, 1024), k);
        k_cross_cols<<<g, 256, 0, st>>>(cells, t0, ctx->cellidx.as<int>(), p, ctx->n2, (int64_t)ctx->n1 * ctx->n2, cp,
                                         cbuf.as<double>());
        KRY_CHECK_LAUNCH();
        SolveInfo si = solve(ctx, e, cbuf.as<double>(), p, sbuf.as<double>(), p, k, rtol, maxit, 0, pre);
        ok = ok && si.converged;
        k_var_final<<<k, 256, 0, st>>>(cbuf.as<double>(), sbuf.as<double>(), p, e->cov.sigma2, var, t0);
        KRY_CHECK_LAUNCH();
    }
    return ok;
}

}  // namespace kry
