// Shared-memory Stockham FFT building blocks (power-of-two lengths).
//
// A length-L transform is run by L / EPT threads, each holding EPT complex
// values in registers per stage.  The stages are Stockham autosort steps
// (the formulation of Govindaraju et al., "High performance discrete Fourier
// transforms on graphics processors", SC 2008): butterfly j of a radix-R stage
// with stride Ns reads x[j + r L/R] (r < R), twiddles them by
// exp(-+2 pi i r (j mod Ns) / (Ns R)), runs an R-point DFT in registers and
// writes x[(j div Ns) Ns R + (j mod Ns) + r Ns].  The buffer is transformed in
// place: every thread reads its inputs, the block synchronises, every thread
// writes, the block synchronises.  One radix-2 or radix-4 stage comes first
// when log2 L is not a multiple of 3; all other stages are radix 8.
//
// Forward transforms use exp(-2 pi i jk / L) and are unscaled; inverse
// transforms use exp(+2 pi i jk / L) and are unscaled too.
#pragma once

#include <cuda_runtime.h>

#include "kry_internal.cuh"

template <typename T> struct cx_of;
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmk(decltype(C().x) a, decltype(C().x) b) {
    C c;
    c.x = a;
    c.y = b;
    return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
    return cmk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by -i (forward) or +i (inverse)
template <typename C, bool INV> __device__ __forceinline__ C cmul_mi(C a) {
    return INV ? cmk<C>(-a.y, a.x) : cmk<C>(a.y, -a.x);
}

// R-point DFTs in registers, sign by INV.
template <typename C, bool INV> __device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <typename C, bool INV> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = cadd(a0, a2), t1 = csub(a0, a2);
    C t2 = cadd(a1, a3), t3 = cmul_mi<C, INV>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <typename C, bool INV> __device__ __forceinline__ void dft8(C* v) {
    using R = decltype(C().x);
    const R h = (R)0.70710678118654752440;
    // even / odd halves
    dft4<C, INV>(v[0], v[2], v[4], v[6]);
    dft4<C, INV>(v[1], v[3], v[5], v[7]);
    // twiddle the odd half by w8^k, w8 = exp(-+2 pi i / 8)
    C o1 = v[3], o2 = v[5], o3 = v[7];
    // w8^1 = h (1 -+ i)
    C w1 = INV ? cmk<C>(h * (o1.x - o1.y), h * (o1.x + o1.y)) : cmk<C>(h * (o1.x + o1.y), h * (o1.y - o1.x));
    // w8^2 = -+ i
    C w2 = cmul_mi<C, INV>(o2);
    // w8^3 = h (-1 -+ i)
    C w3 = INV ? cmk<C>(-h * (o3.x + o3.y), h * (o3.x - o3.y)) : cmk<C>(h * (o3.y - o3.x), -h * (o3.x + o3.y));
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1);
    v[5] = csub(e1, w1);
    v[2] = cadd(e2, w2);
    v[6] = csub(e2, w2);
    v[3] = cadd(e3, w3);
    v[7] = csub(e3, w3);
}

template <typename C, int R, bool INV> __device__ __forceinline__ void dftR(C* v) {
    if constexpr (R == 2) {
        dft2<C, INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<C, INV>(v[0], v[1], v[2], v[3]);
    } else {
        dft8<C, INV>(v);
    }
}

// One Stockham stage on buf[0..L), run by threads t in [0, L/EPT).
template <typename C, int R, bool INV, int EPT>
__device__ __forceinline__ void stockham_stage(C* buf, int L, int Ns, int t, const C* __restrict__ tw) {
    constexpr int NB = EPT / R;
    C v[EPT];
    const int LR = L / R;
    const int LT = L / EPT;
    const int twstep = KRY_TWN / (Ns * R);
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + u * LT;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C x = buf[j + r * LR];
            if (r > 0 && Ns > 1) {
                const C w = tw[r * k * twstep];
                x = INV ? cmulc(x, w) : cmul(x, w);
            }
            v[u * R + r] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        dftR<C, R, INV>(&v[u * R]);
        const int j = t + u * LT;
        const int k = j & (Ns - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[u * R + r];
    }
    __syncthreads();
}

// Full in-place transform of buf[0..L) by the L / EPT threads t of one group.
// Every thread of the block must call this (it synchronises the block).
template <typename C, bool INV, int EPT>
__device__ __forceinline__ void fft_smem(C* buf, int L, int t, const C* __restrict__ tw) {
    int logL = 31 - __clz(L);
    int Ns = 1;
    const int rem = logL % 3;
    if (rem == 1) {
        stockham_stage<C, 2, INV, EPT>(buf, L, 1, t, tw);
        Ns = 2;
    } else if (rem == 2) {
        stockham_stage<C, 4, INV, EPT>(buf, L, 1, t, tw);
        Ns = 4;
    }
    while (Ns < L) {
        stockham_stage<C, 8, INV, EPT>(buf, L, Ns, t, tw);
        Ns *= 8;
    }
}

template <typename T> __device__ __forceinline__ const typename cx_of<T>::type* twiddles(const void* tw32, const void* tw64);
template <> __device__ __forceinline__ const float2* twiddles<float>(const void* tw32, const void*) {
    return static_cast<const float2*>(tw32);
}
template <> __device__ __forceinline__ const double2* twiddles<double>(const void*, const void* tw64) {
    return static_cast<const double2*>(tw64);
}
