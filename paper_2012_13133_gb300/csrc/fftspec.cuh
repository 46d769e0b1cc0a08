// FP32 FFT matvec passes specialised at compile time for one transform
// length L = 2^B and NT transforms per block (B = 6..13, NT = 1, 2, 4, 8).
//
// Same algorithm and data layout as the radix-16 passes of fft16.cuh (Stockham
// stages after Govindaraju et al., SC 2008: radix 2^(B mod 4) first, then
// radix 16; 16 values per thread; transforms interleaved in padded shared
// memory at (pos + (pos >> PS)) * NT + n).  What changes is that every loop
// bound, stride and stage parameter is a constant:
//
//  * Addresses.  A stage's input positions are t + c and its output positions
//    bo(t) + c with c a compile-time constant, and for every stage used here
//    pad(x + c) = pad(x) + pad(c) (pad(x) = x + (x >> PS); c is a multiple of
//    the block of 2^PS positions or cannot carry into it).  Each access is one
//    per-thread base plus an immediate offset.
//  * Twiddles.  Stage s (radix 16, stride Ns > 1) multiplies input m of
//    butterfly k = t mod Ns by W_{16 Ns}^{k m}.  A per-stage table holds the 16
//    twiddles of each k contiguously, row Ns - 1 + k, so a thread's twiddle
//    loads are few 16-byte loads from one 128-byte row (see KRY_KS_TW).
//  * Pruning.  First stages whose upper half of inputs is zero (zero-padded
//    rows and columns, M >= 2n) run half-input DFTs; last stages whose upper
//    half of outputs is discarded (rows >= n1 after the inverse column pass,
//    columns >= n2 after the inverse row pass) compute and store only the
//    lower eight outputs of each radix-16 butterfly.
#pragma once

#include "fft16.cuh"

namespace kspec {

// Pad shift of the interleaved layout (the bank-conflict model of fft16's
// passes: one padding slot every 2^PS positions).
__host__ __device__ constexpr int pad_shift(int L, int NT) {
    return L >= 4096 ? 4 : L == 2048 ? (NT == 1 ? 4 : 3) : NT >= 4 ? 2 : NT == 2 ? 3 : 4;
}

template <int B>
struct Plan {
    static constexpr int L = 1 << B;
    static constexpr int LT = L >> 4;                          // threads per transform
    static constexpr int R0 = (B & 3) ? (1 << (B & 3)) : 16;   // radix of the first stage
    static constexpr int S = (B + 3) >> 2;                     // number of stages
};

// Padded shared-memory offset of position x for NT interleaved transforms.
template <int PS, int NT>
__device__ __forceinline__ int soff(int x) {
    return (x + (x >> PS)) * NT;
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 w, bool conj) {
    return conj ? make_float2(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y)
                : make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// Twiddle scheme of a radix-16 stage (loads are the scarce resource of these
// passes, FP32 arithmetic is not):
//   0: load all 15 twiddles (eight 16-byte loads);
//   1: load W^1..W^4, W^8, W^12 (five 16-byte loads) and form the other nine
//      as one product each;
//   2: load W^1, W^4, W^5 (two 16-byte loads) and form the other twelve with
//      at most two products each (fastest on GB300: 64-vector 1024^2 matvec
//      1.18 / 1.08 / 0.97 ms for schemes 0 / 1 / 2).
#ifndef KRY_KS_TW
#define KRY_KS_TW 2
#endif

// v[m] *= W^{k m} (m = 1..15) from one 16-entry table row (forward twiddles;
// the inverse transform uses their conjugates).
template <bool INV>
__device__ __forceinline__ void twiddle16(float2* v, const float4* __restrict__ row) {
#if KRY_KS_TW == 2
    const float4 a = __ldg(row), c = __ldg(row + 2);
    const float2 w1 = make_float2(a.z, a.w), w4 = make_float2(c.x, c.y), w5 = make_float2(c.z, c.w);
    const float2 w2 = cmulf(w1, w1, false), w3 = cmulf(w4, w1, true), w6 = cmulf(w5, w1, false);
    const float2 w8 = cmulf(w4, w4, false), w9 = cmulf(w4, w5, false), w10 = cmulf(w5, w5, false);
    v[1] = cmulf(v[1], w1, INV);
    v[2] = cmulf(v[2], w2, INV);
    v[3] = cmulf(v[3], w3, INV);
    v[4] = cmulf(v[4], w4, INV);
    v[5] = cmulf(v[5], w5, INV);
    v[6] = cmulf(v[6], w6, INV);
    v[7] = cmulf(v[7], cmulf(w4, w3, false), INV);
    v[8] = cmulf(v[8], w8, INV);
    v[9] = cmulf(v[9], w9, INV);
    v[10] = cmulf(v[10], w10, INV);
    v[11] = cmulf(v[11], cmulf(w5, w6, false), INV);
    v[12] = cmulf(v[12], cmulf(w8, w4, false), INV);
    v[13] = cmulf(v[13], cmulf(w8, w5, false), INV);
    v[14] = cmulf(v[14], cmulf(w10, w4, false), INV);
    v[15] = cmulf(v[15], cmulf(w10, w5, false), INV);
#elif KRY_KS_TW == 1
    const float4 a = __ldg(row), b = __ldg(row + 1), c = __ldg(row + 2), d = __ldg(row + 4), e = __ldg(row + 6);
    const float2 w1 = make_float2(a.z, a.w), w2 = make_float2(b.x, b.y), w3 = make_float2(b.z, b.w);
    const float2 w4 = make_float2(c.x, c.y), w8 = make_float2(d.x, d.y), w12 = make_float2(e.x, e.y);
    v[1] = cmulf(v[1], w1, INV);
    v[2] = cmulf(v[2], w2, INV);
    v[3] = cmulf(v[3], w3, INV);
    v[4] = cmulf(v[4], w4, INV);
    v[5] = cmulf(v[5], cmulf(w4, w1, false), INV);
    v[6] = cmulf(v[6], cmulf(w4, w2, false), INV);
    v[7] = cmulf(v[7], cmulf(w4, w3, false), INV);
    v[8] = cmulf(v[8], w8, INV);
    v[9] = cmulf(v[9], cmulf(w8, w1, false), INV);
    v[10] = cmulf(v[10], cmulf(w8, w2, false), INV);
    v[11] = cmulf(v[11], cmulf(w8, w3, false), INV);
    v[12] = cmulf(v[12], w12, INV);
    v[13] = cmulf(v[13], cmulf(w12, w1, false), INV);
    v[14] = cmulf(v[14], cmulf(w12, w2, false), INV);
    v[15] = cmulf(v[15], cmulf(w12, w3, false), INV);
#else
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 w = __ldg(row + q);
        if (q > 0) v[2 * q] = cmulf(v[2 * q], make_float2(w.x, w.y), INV);
        v[2 * q + 1] = cmulf(v[2 * q + 1], make_float2(w.z, w.w), INV);
    }
#endif
}

// Outputs X[0..7] of a 16-point DFT (4 x 4 as in kry16::dft16; the second
// 4-point DFTs produce only their outputs k2 = 0, 1).  Result in v[0..7].
template <bool INV>
__device__ __forceinline__ void dft16_lo(float2* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<float2, INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    v[5] = cmul(v[5], kry16::w16<float2, INV, 1>());
    v[9] = cmul(v[9], kry16::w16<float2, INV, 2>());
    v[13] = cmul(v[13], kry16::w16<float2, INV, 3>());
    v[6] = cmul(v[6], kry16::w16<float2, INV, 2>());
    v[10] = cmul_mi<float2, INV>(v[10]);
    v[14] = cmul(v[14], kry16::w16<float2, INV, 6>());
    v[7] = cmul(v[7], kry16::w16<float2, INV, 3>());
    v[11] = cmul(v[11], kry16::w16<float2, INV, 6>());
    v[15] = cmul(v[15], kry16::w16<float2, INV, 9>());
    float2 o[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        const float2 a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
        const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
        const float2 t3 = cmul_mi<float2, INV>(csub(a1, a3));
        o[k1] = cadd(t0, t2);       // X[k1]
        o[k1 + 4] = cadd(t1, t3);   // X[k1 + 4]
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = o[k];
}

// One Stockham stage of radix R and stride NS on a length-L transform run by
// L/16 threads; thread t holds the 16/R butterflies j = t + u L/16.
//   ld(c)            value at input position t + c
//   st(bo, c, z)     store z at output position bo + c, bo = (t - k) R + k, k = t mod NS
// HALF_IN: inputs r >= R/2 are zero (first stage, NS = 1).  HALF_OUT: only
// outputs r < 8 are formed and stored (last stage, R = 16).  SYNC: the block
// synchronises between the loads and the stores (in-place shared buffer).
// NOSTORE: outputs stay in registers (slot r = position t + r L/16 for the
// last stage).
template <int L, int R, int NS, bool INV, bool HALF_IN, bool HALF_OUT, bool SYNC, bool NOSTORE, class LD, class ST>
__device__ __forceinline__ void stage(float2* v, int t, const float4* __restrict__ twt, LD&& ld, ST&& st) {
    constexpr int LT = L >> 4, LR = L / R, NB = 16 / R;
    static_assert(NS == 1 || R == 16, "strided stages are radix 16");
    static_assert(!HALF_OUT || (R == 16 && NS == LT), "output pruning is for the last radix-16 stage");
#pragma unroll
    for (int u = 0; u < NB; ++u)
#pragma unroll
        for (int r = 0; r < (HALF_IN ? R / 2 : R); ++r) v[u * R + r] = ld(u * LT + r * LR);
    if constexpr (SYNC) __syncthreads();
    if constexpr (HALF_IN) {
#pragma unroll
        for (int u = 0; u < NB; ++u) kry16::dft_half<float2, R, INV>(v + u * R);
    } else {
        if constexpr (NS > 1) twiddle16<INV>(v, twt + (size_t)(NS - 1 + (t & (NS - 1))) * 8);
        if constexpr (HALF_OUT) {
            dft16_lo<INV>(v);
        } else {
#pragma unroll
            for (int u = 0; u < NB; ++u) kry16::dftR16<float2, R, INV>(v + u * R);
        }
    }
    if constexpr (!NOSTORE) {
        const int k = t & (NS - 1);
        const int bo = (t - k) * R + k;
#pragma unroll
        for (int u = 0; u < NB; ++u)
#pragma unroll
            for (int r = 0; r < (HALF_OUT ? 8 : R); ++r) st(bo, u * LT * R + r * NS, v[u * R + r]);
    }
}

// Stride of stage s.
template <int B>
__host__ __device__ constexpr int stage_ns(int s) {
    return s == 0 ? 1 : Plan<B>::R0 << (4 * (s - 1));
}

// Middle stages 1 .. S-2, in place in shared memory, each followed by a block
// synchronisation.
template <int B, int S_, bool INV, class LDS, class STS>
__device__ __forceinline__ void middle_stages(float2* v, int t, const float4* __restrict__ twt, LDS&& lds, STS&& sts) {
    if constexpr (S_ + 1 < Plan<B>::S) {
        stage<Plan<B>::L, 16, stage_ns<B>(S_), INV, false, false, true, false>(v, t, twt, lds, sts);
        __syncthreads();
        middle_stages<B, S_ + 1, INV>(v, t, twt, lds, sts);
    }
}

}  // namespace kspec
