// Radix-16 register FFT stages for lengths 64 <= L <= 8192.
//
// Each thread holds 16 complex values of one transform.  A transform of
// length L = 2^b runs in ceil(b / 4) Stockham stages (Govindaraju et al.,
// SC 2008 formulation): a first stage of radix 2^(b mod 4) when b is not a
// multiple of 4, then radix-16 stages.  Stage s with radix R and stride Ns
// reads x[j + r L/R], twiddles by exp(-+2 pi i r (j mod Ns) / (Ns R)), runs an
// R-point DFT in registers and writes x[(j - j mod Ns) R + j mod Ns + r Ns];
// thread t owns butterflies j = t + u L/16 (u < 16/R).  After the last stage
// thread t holds positions t + m L/16 (m < 16) in slot m, and the first stage
// of a transform reads exactly those positions, so an inverse transform can
// start from the registers a forward transform ends with (used for the
// eigenvalue multiply of the column pass).
//
// Several transforms share a block, interleaved in shared memory: element
// (pos, n) of transform n lives at (pos + (pos >> PS)) * NT + n, with the
// pad shift PS chosen per length and transform count to avoid bank conflicts.
// Twiddles come from the table W[k] = exp(-2 pi i k / KRY_TWN); radix-8/16
// butterflies load W^1..W^4 (and W^8, W^12) and form the others as one
// product, so each twiddle carries at most ~2 roundings (KRY_TW_DIRECT=1
// loads every twiddle instead).  First stages whose upper half of inputs is known to be
// zero (zero-padded transforms, M >= 2 n) use half-input DFTs.
#pragma once

#include "fft.cuh"

#ifndef KRY_TW_DIRECT
#define KRY_TW_DIRECT 0
#endif

namespace kry16 {

template <typename C> struct Tw16 {
    using R = decltype(C().x);
};

// exp(-+2 pi i m / 16) for compile-time m
template <typename C, bool INV, int M>
__device__ __forceinline__ C w16() {
    using R = decltype(C().x);
    constexpr double c[16] = {1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                              0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                              -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173,
                              0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613};
    constexpr double s[16] = {0.0, 0.38268343236508977173, 0.70710678118654752440, 0.92387953251128675613,
                              1.0, 0.92387953251128675613, 0.70710678118654752440, 0.38268343236508977173,
                              0.0, -0.38268343236508977173, -0.70710678118654752440, -0.92387953251128675613,
                              -1.0, -0.92387953251128675613, -0.70710678118654752440, -0.38268343236508977173};
    // forward: exp(-2 pi i m/16) = cos - i sin
    return cmk<C>((R)c[M & 15], INV ? (R)s[M & 15] : (R)(-s[M & 15]));
}

// 16-point DFT as 4 x 4: v[n2 + 4 n1] -> X[k1 + 4 k2].
template <typename C, bool INV>
__device__ __forceinline__ void dft16(C* v) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<C, INV>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
    // now v[n2 + 4 k1] = Y[n2][k1]; twiddle by W16^(n2 k1)
    v[5] = cmul(v[5], w16<C, INV, 1>());
    v[9] = cmul(v[9], w16<C, INV, 2>());
    v[13] = cmul(v[13], w16<C, INV, 3>());
    v[6] = cmul(v[6], w16<C, INV, 2>());
    v[10] = cmul_mi<C, INV>(v[10]);   // W16^4
    v[14] = cmul(v[14], w16<C, INV, 6>());
    v[7] = cmul(v[7], w16<C, INV, 3>());
    v[11] = cmul(v[11], w16<C, INV, 6>());
    v[15] = cmul(v[15], w16<C, INV, 9>());
    // DFT4 over n2 for each k1: inputs v[4 k1 + n2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<C, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4 x 4 block
    C t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

// R-point DFT whose inputs v[R/2 .. R-1] are zero.
template <typename C, int R, bool INV>
__device__ __forceinline__ void dft_half(C* v) {
    if constexpr (R == 2) {
        v[1] = v[0];
    } else if constexpr (R == 4) {
        const C a0 = v[0], a1 = v[1], b1 = cmul_mi<C, INV>(v[1]);
        v[0] = cadd(a0, a1);
        v[1] = cadd(a0, b1);
        v[2] = csub(a0, a1);
        v[3] = csub(a0, b1);
    } else if constexpr (R == 8) {
        // even part DFT4(a0, a2, 0, 0), odd part DFT4(a1, a3, 0, 0)
        C e[4] = {v[0], v[2], {}, {}}, o[4] = {v[1], v[3], {}, {}};
        dft_half<C, 4, INV>(e);
        dft_half<C, 4, INV>(o);
        v[0] = e[0]; v[2] = e[1]; v[4] = e[2]; v[6] = e[3];
        v[1] = o[0]; v[3] = o[1]; v[5] = o[2]; v[7] = o[3];
        // finish as in dft8: X_k = E_k + w^k O_k, X_{k+4} = E_k - w^k O_k
        using Rt = decltype(C().x);
        const Rt h = (Rt)0.70710678118654752440;
        C o1 = v[3], o2 = v[5], o3 = v[7];
        C w1 = INV ? cmk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cmk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
        C w2 = cmul_mi<C, INV>(o2);
        C w3 = INV ? cmk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cmk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, w1); v[5] = csub(e1, w1);
        v[2] = cadd(e2, w2); v[6] = csub(e2, w2);
        v[3] = cadd(e3, w3); v[7] = csub(e3, w3);
    } else {
        // 4 x 4 with inputs n = n2 + 4 n1, n1 in {0, 1} nonzero
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            C q[4] = {v[n2], v[n2 + 4], {}, {}};
            dft_half<C, 4, INV>(q);
            v[n2] = q[0]; v[n2 + 4] = q[1]; v[n2 + 8] = q[2]; v[n2 + 12] = q[3];
        }
        v[5] = cmul(v[5], w16<C, INV, 1>());
        v[9] = cmul(v[9], w16<C, INV, 2>());
        v[13] = cmul(v[13], w16<C, INV, 3>());
        v[6] = cmul(v[6], w16<C, INV, 2>());
        v[10] = cmul_mi<C, INV>(v[10]);
        v[14] = cmul(v[14], w16<C, INV, 6>());
        v[7] = cmul(v[7], w16<C, INV, 3>());
        v[11] = cmul(v[11], w16<C, INV, 6>());
        v[15] = cmul(v[15], w16<C, INV, 9>());
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4<C, INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
        C t;
        t = v[1]; v[1] = v[4]; v[4] = t;
        t = v[2]; v[2] = v[8]; v[8] = t;
        t = v[3]; v[3] = v[12]; v[12] = t;
        t = v[6]; v[6] = v[9]; v[9] = t;
        t = v[7]; v[7] = v[13]; v[13] = t;
        t = v[11]; v[11] = v[14]; v[14] = t;
    }
}

template <typename C, int R, bool INV>
__device__ __forceinline__ void dftR16(C* v) {
    if constexpr (R == 16) {
        dft16<C, INV>(v);
    } else {
        dftR<C, R, INV>(v);
    }
}

// Multiply v[r] (r = 1..R-1) by W^(r k), W = exp(-+2 pi i / (Ns R)), from the table.
template <typename C, int R, bool INV>
__device__ __forceinline__ void twiddle(C* v, int k, int Ns, const C* __restrict__ tw) {
    if (Ns == 1 || k == 0) return;
    const int ts = (KRY_TWN / (Ns * R)) * k;
    auto ld = [&](int m) {
        C w = tw[m * ts];
        if (INV) w.y = -w.y;
        return w;
    };
    if constexpr (R == 2) {
        v[1] = cmul(v[1], ld(1));
    } else if constexpr (R == 4) {
        v[1] = cmul(v[1], ld(1));
        v[2] = cmul(v[2], ld(2));
        v[3] = cmul(v[3], ld(3));
    } else {
#if KRY_TW_DIRECT
#pragma unroll
        for (int m = 1; m < R; ++m) v[m] = cmul(v[m], ld(m));
#else
        // R = 8 or 16: load W^1..W^4 (and W^8, W^12) and form the rest as one
        // product W^(4a) W^b (at most ~2 roundings per twiddle)
        const C w1 = ld(1), w2 = ld(2), w3 = ld(3), w4 = ld(4);
        v[1] = cmul(v[1], w1);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], cmul(w4, w1));
        v[6] = cmul(v[6], cmul(w4, w2));
        v[7] = cmul(v[7], cmul(w4, w3));
        if constexpr (R == 16) {
            const C w8 = ld(8), w12 = ld(12);
            v[8] = cmul(v[8], w8);
            v[9] = cmul(v[9], cmul(w8, w1));
            v[10] = cmul(v[10], cmul(w8, w2));
            v[11] = cmul(v[11], cmul(w8, w3));
            v[12] = cmul(v[12], w12);
            v[13] = cmul(v[13], cmul(w12, w1));
            v[14] = cmul(v[14], cmul(w12, w2));
            v[15] = cmul(v[15], cmul(w12, w3));
        }
#endif
    }
}

// Butterflies of one stage on the 16 values a thread holds: 16/R butterflies,
// slot u*R + r holds input r of butterfly j = t + u L/16.
template <typename C, int R, bool INV>
__device__ __forceinline__ void butterflies(C* v, int t, int LT, int Ns, const C* __restrict__ tw) {
#pragma unroll
    for (int u = 0; u < 16 / R; ++u) {
        const int j = t + u * LT;
        twiddle<C, R, INV>(v + u * R, j & (Ns - 1), Ns, tw);
        dftR16<C, R, INV>(v + u * R);
    }
}

// Input position of slot (u, r) and output position of slot (u, r) for a stage.
__device__ __forceinline__ int in_pos(int t, int u, int r, int LT, int LR) { return t + u * LT + r * LR; }
__device__ __forceinline__ int out_pos(int t, int u, int r, int LT, int R, int Ns) {
    const int j = t + u * LT;
    const int k = j & (Ns - 1);
    return (j - k) * R + k + r * Ns;
}

// Radix of stage s for L = 2^b.
__device__ __forceinline__ int stage_radix(int b, int s) {
    const int r0 = b & 3;
    return (s == 0 && r0) ? (1 << r0) : 16;
}
__device__ __forceinline__ int num_stages(int b) { return (b + 3) >> 2; }

// Shared-memory position of element pos of transform n (NT transforms interleaved).
__device__ __forceinline__ int spos(int pos, int PS, int NT, int n) { return (pos + (pos >> PS)) * NT + n; }

// One stage: load 16 values with LD(pos) (pos = input position), butterflies,
// store with ST(pos, value).  If IN_PLACE, the block synchronises between the
// loads and the stores (all reads of the shared buffer finish first).
template <typename C, int R, bool INV, class LD, class ST, bool HALF = false>
__device__ __forceinline__ void stage(C* v, int t, int L, int Ns, const C* __restrict__ tw, LD&& ld, ST&& st,
                                      bool in_place) {
    const int LT = L >> 4, LR = L / R;
#pragma unroll
    for (int u = 0; u < 16 / R; ++u)
#pragma unroll
        for (int r = 0; r < (HALF ? R / 2 : R); ++r) v[u * R + r] = ld(in_pos(t, u, r, LT, LR));
    if (in_place) __syncthreads();
    if constexpr (HALF) {
        // first stage (Ns = 1): no twiddles; inputs r >= R/2 lie at positions >= L/2, which are zero
#pragma unroll
        for (int u = 0; u < 16 / R; ++u) dft_half<C, R, INV>(v + u * R);
    } else {
        butterflies<C, R, INV>(v, t, LT, Ns, tw);
    }
#pragma unroll
    for (int u = 0; u < 16 / R; ++u)
#pragma unroll
        for (int r = 0; r < R; ++r) st(out_pos(t, u, r, LT, R, Ns), v[u * R + r]);
}

// A whole transform of length L = 2^b (b >= 6, so at least two stages): the
// first stage (runtime radix) loads with LD0 and stores to shared memory with
// STS, the middle radix-16 stages work in shared memory (LDS/STS, in place),
// the last radix-16 stage loads with LDS and stores with STL.  The block is
// synchronised after every shared-memory store phase.  FIRST_IN_PLACE tells
// whether LD0 reads the same shared buffer that STS writes.
template <typename C, bool INV, bool HALF0 = false, class LD0, class LDS, class STS, class STL>
__device__ __forceinline__ void transform(int b, C* v, int t, const C* __restrict__ tw, LD0&& ld0, LDS&& lds,
                                          STS&& sts, STL&& stl, bool first_in_place, bool last_in_place) {
    const int L = 1 << b;
    const int nst = num_stages(b);
    const int r0 = stage_radix(b, 0);
    switch (r0) {
        case 2: stage<C, 2, INV, LD0&, STS&, HALF0>(v, t, L, 1, tw, ld0, sts, first_in_place); break;
        case 4: stage<C, 4, INV, LD0&, STS&, HALF0>(v, t, L, 1, tw, ld0, sts, first_in_place); break;
        case 8: stage<C, 8, INV, LD0&, STS&, HALF0>(v, t, L, 1, tw, ld0, sts, first_in_place); break;
        default: stage<C, 16, INV, LD0&, STS&, HALF0>(v, t, L, 1, tw, ld0, sts, first_in_place); break;
    }
    __syncthreads();
    int Ns = r0;
#pragma unroll 1
    for (int s = 1; s < nst - 1; ++s) {
        stage<C, 16, INV>(v, t, L, Ns, tw, lds, sts, true);
        __syncthreads();
        Ns *= 16;
    }
    stage<C, 16, INV>(v, t, L, Ns, tw, lds, stl, last_in_place);
}

// Runtime-radix dispatch of one stage.
template <typename C, bool INV, class LD, class ST>
__device__ __forceinline__ void stage_any(int R, C* v, int t, int L, int Ns, const C* __restrict__ tw, LD&& ld,
                                          ST&& st, bool in_place) {
    switch (R) {
        case 2: stage<C, 2, INV>(v, t, L, Ns, tw, ld, st, in_place); break;
        case 4: stage<C, 4, INV>(v, t, L, Ns, tw, ld, st, in_place); break;
        case 8: stage<C, 8, INV>(v, t, L, Ns, tw, ld, st, in_place); break;
        default: stage<C, 16, INV>(v, t, L, Ns, tw, ld, st, in_place); break;
    }
}

// Variant of the last stage that leaves its outputs in registers, slot m =
// position t + m L/16 (the last stage always has radix 16 for L >= 64, one
// butterfly per thread, so slot r already is position t + r L/16).
template <typename C, bool INV, class LD>
__device__ __forceinline__ void last_stage_regs(C* v, int t, int L, int Ns, const C* __restrict__ tw, LD&& ld,
                                                bool in_place) {
    const int LT = L >> 4;
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ld(t + r * LT);
    if (in_place) __syncthreads();
    twiddle<C, 16, INV>(v, t & (Ns - 1), Ns, tw);
    dft16<C, INV>(v);
}

// First stage fed from registers holding positions t + m L/16 in slot m
// (radix R, Ns = 1): slot (u, r) of the stage reads position t + (u + r 16/R) L/16.
template <typename C, bool INV, class ST>
__device__ __forceinline__ void first_stage_regs(int R, C* v, int t, int L, const C* __restrict__ tw, ST&& st) {
    C w[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) w[m] = v[m];
    switch (R) {
        case 2:
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int r = 0; r < 2; ++r) v[u * 2 + r] = w[u + r * 8];
            butterflies<C, 2, INV>(v, t, L >> 4, 1, tw);
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int r = 0; r < 2; ++r) st(out_pos(t, u, r, L >> 4, 2, 1), v[u * 2 + r]);
            break;
        case 4:
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int r = 0; r < 4; ++r) v[u * 4 + r] = w[u + r * 4];
            butterflies<C, 4, INV>(v, t, L >> 4, 1, tw);
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int r = 0; r < 4; ++r) st(out_pos(t, u, r, L >> 4, 4, 1), v[u * 4 + r]);
            break;
        case 8:
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int r = 0; r < 8; ++r) v[u * 8 + r] = w[u + r * 2];
            butterflies<C, 8, INV>(v, t, L >> 4, 1, tw);
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int r = 0; r < 8; ++r) st(out_pos(t, u, r, L >> 4, 8, 1), v[u * 8 + r]);
            break;
        default:
            butterflies<C, 16, INV>(v, t, L >> 4, 1, tw);
#pragma unroll
            for (int r = 0; r < 16; ++r) st(out_pos(t, 0, r, L >> 4, 16, 1), v[r]);
            break;
    }
}

}  // namespace kry16
