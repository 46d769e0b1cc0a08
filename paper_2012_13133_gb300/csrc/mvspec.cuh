// The three FP32 matvec passes (Sec. 3: K v = A F^-1 (Lambda . F (A^T v)) +
// tau^2 v on the circulant embedding) specialised for transform length
// L = 2^B and NT transforms per block; see fftspec.cuh.  Each translation
// unit mvspec_{a,b,c}.cu instantiates one pass for every supported (B, NT)
// and exposes a runtime dispatcher; matvec.cu calls them for FP32 batches.
//
// Layouts (identical to the generic radix-16 passes, so the two can be mixed):
//  * slab: per complex pair an n1 x M2 complex intermediate, stored in column
//    tiles slab[pair][tile][i][c], c < C, tile = column / C;
//  * lamP: eigenvalues transposed to [M2][M1], scaled by 1 / (M1 M2), each
//    column permuted so that row t + m L/16 sits at 16 t + m;
//  * twt: stage twiddle table, row Ns - 1 + k (Ns a power of two <= 512,
//    k < Ns) holds W_{16 Ns}^{k m}, m = 0..15, W_n = exp(-2 pi i / n).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"
#include "fftspec.cuh"
#include "kry_internal.cuh"

#ifndef KRY_KS_MAXREG
#define KRY_KS_MAXREG 64   // register cap per thread of the specialised passes
#endif

namespace kspec {

constexpr int tpb(int B, int NT) { return NT * ((1 << B) >> 4); }
// Minimum resident blocks per SM that caps registers at KRY_KS_MAXREG (at most
// 32, the SM's block limit; tiny blocks are then capped less tightly).
constexpr int minb(int B, int NT) {
    return 65536 / (KRY_KS_MAXREG * tpb(B, NT)) < 1    ? 1
           : 65536 / (KRY_KS_MAXREG * tpb(B, NT)) > 32 ? 32
                                                       : 65536 / (KRY_KS_MAXREG * tpb(B, NT));
}

// Shared-memory bytes of a block.
constexpr size_t smem_bytes(int B, int NT) {
    return (size_t)((1 << B) + ((1 << B) >> pad_shift(1 << B, NT))) * NT * sizeof(float2);
}

// ---------------------------------------------------------------- pass A
// Scatter the observed values of NT rows (two real vectors as re/im) into
// zeroed rows, forward row FFT (half-input first stage: columns >= n2 are
// zero), store the n1 x M2 slab in column tiles of width C (C <= L/16).
template <int B, int NT>
__global__ void __launch_bounds__(tpb(B, NT), minb(B, NT))
    ks_pass_a(const float* __restrict__ vin, int64_t ld, const double* __restrict__ scale, int nvec, int pair0,
              const int* __restrict__ rowptr, const int* __restrict__ colidx, int n1, int n2, int C, int logC,
              float2* __restrict__ slab, const float4* __restrict__ twt, const int* __restrict__ skip) {
    using P = Plan<B>;
    constexpr int L = P::L, LT = P::LT, PS = pad_shift(L, NT);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();   // the vectors and skip flags come from the kernel before
    pdl_launch_dependents();
    const int n = threadIdx.x & (NT - 1), t = threadIdx.x / NT;
    const int row = blockIdx.x * NT + n;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;
    if (skip && skip[va] && (!has_b || skip[vb])) return;   // both columns finished (whole block)
    float2* sb = reinterpret_cast<float2*>(smem_raw) + n;
    const float2 zero = make_float2(0.f, 0.f);
    const int tb = soff<PS, NT>(t);

    // The row's observed cells are loaded into registers first (a row holds at
    // most n2 <= L/2 = 8 L/16 of them, so a fixed-trip predicated loop covers
    // it), and their latency overlaps the zero fill.
    int col[8];
    float2 val[8];
    if (row < n1) {
        const float sa = scale ? (float)scale[va] : 1.f;
        const float sbv = (scale && has_b) ? (float)scale[vb] : 1.f;
        const int q0 = rowptr[row] + t, q1 = rowptr[row + 1];
        const float* pa = vin + (int64_t)va * ld;
        const float* pb = vin + (int64_t)vb * ld;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = q0 + i * LT;
            col[i] = q < q1 ? colidx[q] : -1;
            val[i] = q < q1 ? make_float2(pa[q] * sa, has_b ? pb[q] * sbv : 0.f) : zero;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) col[i] = -1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)   // positions t + i L/16 cover [0, L/2), which holds [0, n2)
        if (t + i * LT < n2) sb[tb + soff<PS, NT>(i * LT)] = zero;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i)
        if (col[i] >= 0) sb[soff<PS, NT>(col[i])] = val[i];
    __syncthreads();

    // global store of output position p = t + c (c a multiple of L/16 >= C)
    const int64_t tstride = (int64_t)n1 * C;
    float2* out = slab + (int64_t)blockIdx.y * n1 * (int64_t)(L) + (int64_t)row * C +
                  (int64_t)(t >> logC) * tstride + (t & (C - 1));
    const int64_t gstep = (int64_t)(LT >> logC) * tstride;
    const bool live = row < n1;

    auto ld0 = [&](int c) { return (t + c < n2) ? sb[tb + soff<PS, NT>(c)] : zero; };
    auto lds = [&](int c) { return sb[tb + soff<PS, NT>(c)]; };
    auto sts = [&](int bo, int c, float2 z) { sb[soff<PS, NT>(bo) + soff<PS, NT>(c)] = z; };
    auto stg = [&](int, int c, float2 z) {
        if (live) out[(c / LT) * gstep] = z;
    };
    float2 v[16];
    stage<L, P::R0, 1, false, true, false, true, false>(v, t, twt, ld0, sts);
    __syncthreads();
    middle_stages<B, 1, false>(v, t, twt, lds, sts);
    stage<L, 16, LT, false, false, false, false, false>(v, t, twt, lds, stg);
}

// ---------------------------------------------------------------- pass B
// Per column (NT columns = one slab tile per block): forward column FFT
// (half-input: rows >= n1 are zero) ending in registers, multiply by Lambda,
// inverse column FFT starting from registers, keep rows < n1.
template <int B, int NT>
__global__ void __launch_bounds__(tpb(B, NT), minb(B, NT))
    ks_pass_b(float2* __restrict__ slab, const float* __restrict__ lamP, int n1, int M2,
              const float4* __restrict__ twt, int pair0, int64_t lam_stride, int vpt, const int* __restrict__ skip,
              int nvec) {
    using P = Plan<B>;
    constexpr int L = P::L, LT = P::LT, PS = pad_shift(L, NT);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    pdl_wait();   // the slab comes from pass A
    pdl_launch_dependents();
    if (skip) {
        const int va = 2 * (pair0 + (int)blockIdx.y), vb = va + 1;
        if (skip[va] && (vb >= nvec || skip[vb])) return;
    }
    const int c = threadIdx.x & (NT - 1), t = threadIdx.x / NT;
    const int tile = blockIdx.x;
    float2* sb = reinterpret_cast<float2*>(smem_raw) + c;
    float2* blk = slab + (int64_t)blockIdx.y * n1 * M2 + (int64_t)tile * n1 * NT + (int64_t)t * NT + c;
    const float2 zero = make_float2(0.f, 0.f);
    const int tb = soff<PS, NT>(t);

    auto ldg = [&](int cc) { return (t + cc < n1) ? blk[cc * NT] : zero; };
    auto lds = [&](int cc) { return sb[tb + soff<PS, NT>(cc)]; };
    auto sts = [&](int bo, int cc, float2 z) { sb[soff<PS, NT>(bo) + soff<PS, NT>(cc)] = z; };
    auto none = [&](int, int, float2) {};
    auto stg = [&](int, int cc, float2 z) {
        if (t + cc < n1) blk[cc * NT] = z;
    };
    float2 v[16];
    // forward, ending with slot m = row t + m L/16
    stage<L, P::R0, 1, false, true, false, false, false>(v, t, twt, ldg, sts);
    __syncthreads();
    middle_stages<B, 1, false>(v, t, twt, lds, sts);
    stage<L, 16, LT, false, false, false, true, true>(v, t, twt, lds, none);

    // eigenvalue multiply
    const int theta = vpt ? (2 * (pair0 + (int)blockIdx.y)) / vpt : 0;
    // column-permuted eigenvalues: slot m of thread t at 16 t + m
    const float4* lam = reinterpret_cast<const float4*>(lamP + theta * lam_stride + (int64_t)(tile * NT + c) * L) + 4 * t;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 l = __ldg(lam + q);
        v[4 * q] = make_float2(v[4 * q].x * l.x, v[4 * q].y * l.x);
        v[4 * q + 1] = make_float2(v[4 * q + 1].x * l.y, v[4 * q + 1].y * l.y);
        v[4 * q + 2] = make_float2(v[4 * q + 2].x * l.z, v[4 * q + 2].y * l.z);
        v[4 * q + 3] = make_float2(v[4 * q + 3].x * l.w, v[4 * q + 3].y * l.w);
    }

    // inverse, first stage fed from registers: input position t + c lives in slot c / (L/16)
    float2 w[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) w[m] = v[m];
    auto ldr = [&](int cc) { return w[cc / LT]; };
    stage<L, P::R0, 1, true, false, false, false, false>(v, t, twt, ldr, sts);
    __syncthreads();
    middle_stages<B, 1, true>(v, t, twt, lds, sts);
    stage<L, 16, LT, true, false, true, false, false>(v, t, twt, lds, stg);
}

// ---------------------------------------------------------------- pass C
// Inverse row FFT of NT slab rows (last stage keeps columns < n2), gather the
// observed cells, add the nugget, write K v, and (dots != NULL) per-block FP64
// partials of v . K v.
template <int B, int NT>
__global__ void __launch_bounds__(tpb(B, NT), minb(B, NT))
    ks_pass_c(const float2* __restrict__ slab, const float* __restrict__ vin, int64_t ld_in,
              const double* __restrict__ scale, float* __restrict__ vout, int64_t ld_out, int nvec, int pair0,
              const int* __restrict__ rowptr, const int* __restrict__ colidx, int n1, int n2, int C, int logC,
              double tau2, double* __restrict__ dots, int ndot_stride, const float4* __restrict__ twt,
              const double* __restrict__ tau2v, int vpt, const int* __restrict__ skip) {
    using P = Plan<B>;
    constexpr int L = P::L, LT = P::LT, PS = pad_shift(L, NT);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[2][32];
    pdl_wait();   // the slab comes from pass B
    pdl_launch_dependents();
    const int n = threadIdx.x & (NT - 1), t = threadIdx.x / NT;
    const int row = blockIdx.x * NT + n;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;
    if (skip && skip[va] && (!has_b || skip[vb])) return;   // both columns finished (whole block)
    float2* sb = reinterpret_cast<float2*>(smem_raw) + n;
    const float2 zero = make_float2(0.f, 0.f);
    const int tb = soff<PS, NT>(t);
    const bool live = row < n1;
    const int q0 = live ? rowptr[row] + t : 0, q1 = live ? rowptr[row + 1] : 0;   // read early

    const int64_t tstride = (int64_t)n1 * C;
    const float2* in = slab + (int64_t)blockIdx.y * n1 * (int64_t)(L) + (int64_t)row * C +
                       (int64_t)(t >> logC) * tstride + (t & (C - 1));
    const int64_t gstep = (int64_t)(LT >> logC) * tstride;
    auto ldg = [&](int c) { return live ? in[(c / LT) * gstep] : zero; };
    auto lds = [&](int c) { return sb[tb + soff<PS, NT>(c)]; };
    auto sts = [&](int bo, int c, float2 z) { sb[soff<PS, NT>(bo) + soff<PS, NT>(c)] = z; };
    auto stn = [&](int, int c, float2 z) {
        if (t + c < n2) sb[tb + soff<PS, NT>(c)] = z;
    };
    float2 v[16];
    stage<L, P::R0, 1, true, false, false, false, false>(v, t, twt, ldg, sts);
    __syncthreads();
    middle_stages<B, 1, true>(v, t, twt, lds, sts);
    stage<L, 16, LT, true, false, true, true, false>(v, t, twt, lds, stn);
    __syncthreads();

    kry::DotAcc<float> acc_a, acc_b;
    if (live) {
        const float sa = scale ? (float)scale[va] : 1.f;
        const float sbv = (scale && has_b) ? (float)scale[vb] : 1.f;
        const float t2 = (float)(tau2v ? tau2v[vpt ? va / vpt : 0] : tau2);
        const float* pa = vin + (int64_t)va * ld_in;
        const float* pb = vin + (int64_t)vb * ld_in;
        float* oa = vout + (int64_t)va * ld_out;
        float* ob = vout + (int64_t)vb * ld_out;
        // at most n2 <= 8 L/16 cells per row: fixed-trip predicated loop
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = q0 + i * LT;
            if (q < q1) {
                const float2 z = sb[soff<PS, NT>(colidx[q])];
                const float xa = pa[q] * sa;
                const float ya = z.x + t2 * xa;
                oa[q] = ya;
                acc_a.add_prod(xa, ya);
                if (has_b) {
                    const float xb = pb[q] * sbv;
                    const float yb = z.y + t2 * xb;
                    ob[q] = yb;
                    acc_b.add_prod(xb, yb);
                }
            }
        }
    }
    if (dots != nullptr) {
        double da = acc_a.value(), db = acc_b.value();
        // fixed-order block reduction (rows interleaved across lanes, n fastest)
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (blockDim.x >= 32) {
            for (int o = 16; o > 0; o >>= 1) {
                da += __shfl_down_sync(0xffffffffu, da, o);
                db += __shfl_down_sync(0xffffffffu, db, o);
            }
            if (lane == 0) {
                red[0][w] = da;
                red[1][w] = db;
            }
        } else {
            red[0][threadIdx.x] = da;
            red[1][threadIdx.x] = db;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s0 = 0.0, s1 = 0.0;
            const int nw = (blockDim.x >= 32) ? (blockDim.x >> 5) : blockDim.x;
            for (int k = 0; k < nw; ++k) {
                s0 += red[0][k];
                s1 += red[1][k];
            }
            dots[(int64_t)va * ndot_stride + blockIdx.x] = s0;
            if (has_b) dots[(int64_t)vb * ndot_stride + blockIdx.x] = s1;
        }
    }
}

// ---------------------------------------------------------------- dispatch

// Arguments of one specialised matvec pass triple (per batch of pairs).
struct SpecArgs {
    const float* vin;
    int64_t ld_in;
    const double* scale;
    float* vout;
    int64_t ld_out;
    int nvec, pair0, np;
    const int* rowptr;
    const int* colidx;
    int n1, n2, M1, M2;
    int G, C, logC;
    float2* slab;
    const float* lamP;   // column-permuted FP32 eigenvalues (kry_embed::lam32P)
    int64_t lam_stride;
    int vpt;
    double tau2;
    const double* tau2v;
    double* dots;
    int nds;
    const float4* twt;
    const int* skip;
};

// True if the specialised kernels cover this shape: 64 <= M <= 8192, rows and
// columns per block in {1, 2, 4, 8} within 1024 threads, slab tile width C
// at most M2 / 16.
bool supported(int M1, int M2, int G, int C);

// Launch pass A, B or C (returns false if the (B, NT) pair is not compiled).
bool launch_a(const SpecArgs& a, cudaStream_t st);
bool launch_b(const SpecArgs& a, cudaStream_t st);
bool launch_c(const SpecArgs& a, cudaStream_t st);

// Stage twiddle table of 1023 rows x 16 complex FP32 values (see above).
constexpr int TWT_ROWS = 1023;
void fill_stage_twiddles(float2* twt_dev, cudaStream_t st);

}  // namespace kspec

namespace kspec {

// Calls f.template run<B, NT>() for a runtime (B, NT) with 6 <= B <= 13,
// NT in {1, 2, 4, 8} and at most 1024 threads per block; false otherwise.
template <int B, class F>
bool dispatch_nt(int nt, const F& f) {
    switch (nt) {
        case 1: return f.template run<B, 1>();
        case 2: return f.template run<B, 2>();
        case 4:
            if constexpr (tpb(B, 4) <= 1024) return f.template run<B, 4>();
            return false;
        case 8:
            if constexpr (tpb(B, 8) <= 1024) return f.template run<B, 8>();
            return false;
        default: return false;
    }
}

template <class F>
bool dispatch(int b, int nt, const F& f) {
    switch (b) {
        case 6: return dispatch_nt<6>(nt, f);
        case 7: return dispatch_nt<7>(nt, f);
        case 8: return dispatch_nt<8>(nt, f);
        case 9: return dispatch_nt<9>(nt, f);
        case 10: return dispatch_nt<10>(nt, f);
        case 11: return dispatch_nt<11>(nt, f);
        case 12: return dispatch_nt<12>(nt, f);
        case 13: return dispatch_nt<13>(nt, f);
        default: return false;
    }
}

inline int ilog2i(int x) { return 31 - __builtin_clz((unsigned)x); }

}  // namespace kspec
