// BTTB covariance matvec by circulant embedding (Sec. 3: Sigma is symmetric
// BTTB, stored through one row and applied in O(n log n) with FFTs; the
// embedding's eigenvalues diagonalise it, Appendix A Eq. circ_diag):
//
//   K v = A F^-1 ( Lambda .* F ( A^T v ) ) + tau^2 v
//
// on the M1 x M2 torus, A the observation mask.  Two real vectors travel as
// the real and imaginary parts of one complex field; that is exact because
// Lambda is real and even.  The 2-D transform is split into three kernels:
//
//   pass A  per grid row i < n1: scatter the observed values of the row into
//           a zero row of length M2 in shared memory, forward FFT, store the
//           row into the intermediate slab (n1 x M2 complex per pair);
//   pass B  per tile of C columns: load the n1 nonzero rows of each column,
//           forward FFT of length M1, multiply by Lambda (scaled by
//           1/(M1 M2)), inverse FFT, store the first n1 rows back;
//   pass C  per grid row: inverse FFT of length M2, gather the observed
//           columns, add the nugget term, and (optionally) accumulate the
//           FP64 dot product of input and output for the Krylov loops.
//
// The slab is laid out in column tiles, slab[pair][tile][i][c] with
// c < C, so that pass B reads and writes one contiguous block per CTA and
// passes A and C touch G*C contiguous elements per tile for G rows per CTA.
#include <algorithm>
#include <mutex>
#include <string>

#include "dfloat.cuh"
#include "fft.cuh"
#include "fft16.cuh"
#include "mvspec.cuh"
#include "kry_internal.cuh"

namespace kry {

// ------------------------------------------------------------------ pass A

template <typename T, int EPT, int G>
__global__ void __launch_bounds__(EPT >= 16 ? 512 : 1024) k_pass_a(const T* __restrict__ vin, int64_t ld, const double* __restrict__ scale,
                                                 int nvec, int pair0, const int* __restrict__ rowptr,
                                                 const int* __restrict__ colidx, int n1, int M2, int C,
                                                 typename cx_of<T>::type* __restrict__ slab, const void* tw32,
                                                 const void* tw64) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    const int L = M2;
    const int stride = L + 1;
    const int LT = L / EPT;
    const int g = threadIdx.x / LT;
    const int tl = threadIdx.x - g * LT;
    const int row0 = blockIdx.x * G;
    const int row = row0 + g;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;
    Cx* rb = buf + g * stride;

    for (int k = tl; k < L; k += LT) rb[k] = cmk<Cx>((T)0, (T)0);
    __syncthreads();
    if (row < n1) {
        const T sa = scale ? (T)scale[va] : (T)1;
        const T sb = (scale && has_b) ? (T)scale[vb] : (T)1;
        const T* pa = vin + (int64_t)va * ld;
        const T* pb = vin + (int64_t)vb * ld;
        const int q1 = rowptr[row + 1];
        for (int q = rowptr[row] + tl; q < q1; q += LT) {
            const int c = colidx[q];
            const T a = pa[q] * sa;
            const T b = has_b ? pb[q] * sb : (T)0;
            rb[c] = cmk<Cx>(a, b);
        }
    }
    __syncthreads();
    fft_smem<Cx, false, EPT>(rb, L, tl, twiddles<T>(tw32, tw64));

    // store: slab[pair][tile][row][c]
    Cx* out = slab + (int64_t)blockIdx.y * n1 * M2;
    const int GC = G * C;
    for (int e = threadIdx.x; e < G * L; e += blockDim.x) {
        const int tile = e / GC;
        const int rem = e - tile * GC;
        const int gg = rem / C;
        const int c = rem - gg * C;
        const int r = row0 + gg;
        if (r < n1) out[(int64_t)tile * n1 * C + (int64_t)r * C + c] = buf[gg * stride + tile * C + c];
    }
}

// ------------------------------------------------------------------ pass B

template <typename T, int EPT, int CC>
__global__ void __launch_bounds__(EPT >= 16 ? 512 : 1024) k_pass_b(typename cx_of<T>::type* __restrict__ slab, const T* __restrict__ lamT,
                                                 int n1, int M1, int M2, const void* tw32, const void* tw64,
                                                 int pair0, int64_t lam_stride, int vpt) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    const int L = M1;
    const int stride = L + 1;
    const int LT = L / EPT;
    const int g = threadIdx.x / LT;
    const int tl = threadIdx.x - g * LT;
    const int tile = blockIdx.x;
    Cx* blk = slab + (int64_t)blockIdx.y * n1 * M2 + (int64_t)tile * n1 * CC;

    const int nload = n1 * CC;
    for (int e = threadIdx.x; e < nload; e += blockDim.x) {
        const int i = e / CC;
        const int c = e - i * CC;
        buf[c * stride + i] = blk[e];
    }
    for (int e = threadIdx.x; e < (L - n1) * CC; e += blockDim.x) {
        const int c = e / (L - n1);
        const int i = n1 + (e - c * (L - n1));
        buf[c * stride + i] = cmk<Cx>((T)0, (T)0);
    }
    __syncthreads();
    Cx* cb = buf + g * stride;
    const Cx* tw = twiddles<T>(tw32, tw64);
    fft_smem<Cx, false, EPT>(cb, L, tl, tw);
    const int theta = vpt ? (2 * (pair0 + (int)blockIdx.y)) / vpt : 0;
    const T* lam = lamT + theta * lam_stride + (int64_t)(tile * CC + g) * L;
    for (int k = tl; k < L; k += LT) {
        const T l = lam[k];
        Cx z = cb[k];
        cb[k] = cmk<Cx>(z.x * l, z.y * l);
    }
    __syncthreads();
    fft_smem<Cx, true, EPT>(cb, L, tl, tw);
    for (int e = threadIdx.x; e < nload; e += blockDim.x) {
        const int i = e / CC;
        const int c = e - i * CC;
        blk[e] = buf[c * stride + i];
    }
}

// ------------------------------------------------------------------ pass C

// MODE 0: gather the observed cells, add tau2 * (scaled input), optional dot.
// MODE 1: write every grid cell (n1 x n2 row-major) per vector, no nugget.
template <typename T, int EPT, int G, int MODE>
__global__ void __launch_bounds__(EPT >= 16 ? 512 : 1024) k_pass_c(const typename cx_of<T>::type* __restrict__ slab, const T* __restrict__ vin,
                                                 int64_t ld_in, const double* __restrict__ scale, T* __restrict__ vout,
                                                 int64_t ld_out, int nvec, int pair0, const int* __restrict__ rowptr,
                                                 const int* __restrict__ colidx, int n1, int n2, int M2, int C,
                                                 double tau2, double* __restrict__ dots, int ndot_stride,
                                                 const void* tw32, const void* tw64, const double* __restrict__ tau2v,
                                                 int vpt) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    __shared__ double red[2][32];
    const int L = M2;
    const int stride = L + 1;
    const int LT = L / EPT;
    const int g = threadIdx.x / LT;
    const int tl = threadIdx.x - g * LT;
    const int row0 = blockIdx.x * G;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;

    const Cx* in = slab + (int64_t)blockIdx.y * n1 * M2;
    const int GC = G * C;
    for (int e = threadIdx.x; e < G * L; e += blockDim.x) {
        const int tile = e / GC;
        const int rem = e - tile * GC;
        const int gg = rem / C;
        const int c = rem - gg * C;
        const int r = row0 + gg;
        buf[gg * stride + tile * C + c] =
            (r < n1) ? in[(int64_t)tile * n1 * C + (int64_t)r * C + c] : cmk<Cx>((T)0, (T)0);
    }
    __syncthreads();
    Cx* rb = buf + g * stride;
    fft_smem<Cx, true, EPT>(rb, L, tl, twiddles<T>(tw32, tw64));

    const int row = row0 + g;
    DotAcc<T> acc_a, acc_b;
    if (row < n1) {
        if (MODE == 0) {
            const T sa = scale ? (T)scale[va] : (T)1;
            const T sb = (scale && has_b) ? (T)scale[vb] : (T)1;
            const T t2 = (T)(tau2v ? tau2v[vpt ? va / vpt : 0] : tau2);
            const T* pa = vin + (int64_t)va * ld_in;
            const T* pb = vin + (int64_t)vb * ld_in;
            T* oa = vout + (int64_t)va * ld_out;
            T* ob = vout + (int64_t)vb * ld_out;
            const int q1 = rowptr[row + 1];
            for (int q = rowptr[row] + tl; q < q1; q += LT) {
                const Cx z = rb[colidx[q]];
                const T xa = pa[q] * sa;
                const T ya = z.x + t2 * xa;
                oa[q] = ya;
                acc_a.add_prod(xa, ya);
                if (has_b) {
                    const T xb = pb[q] * sb;
                    const T yb = z.y + t2 * xb;
                    ob[q] = yb;
                    acc_b.add_prod(xb, yb);
                }
            }
        } else {
            T* oa = vout + (int64_t)va * ld_out + (int64_t)row * n2;
            T* ob = vout + (int64_t)vb * ld_out + (int64_t)row * n2;
            for (int j = tl; j < n2; j += LT) {
                const Cx z = rb[j];
                oa[j] = z.x;
                if (has_b) ob[j] = z.y;
            }
        }
    }
    if (MODE == 0 && dots != nullptr) {
        double da = acc_a.value(), db = acc_b.value();
        // block reduction of (da, db) in a fixed order; blocks narrower than a
        // warp (short rows) reduce serially through shared memory
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
            double sa = 0.0, sb = 0.0;
            const int nw = (blockDim.x >= 32) ? (blockDim.x >> 5) : blockDim.x;
            for (int k = 0; k < nw; ++k) {
                sa += red[0][k];
                sb += red[1][k];
            }
            dots[(int64_t)va * ndot_stride + blockIdx.x] = sa;
            if (has_b) dots[(int64_t)vb * ndot_stride + blockIdx.x] = sb;
        }
    }
}

// ------------------------------------------------------------------ radix-16 passes (64 <= L <= 8192)

#ifndef KRY_K16_MINB
#define KRY_K16_MINB 2   // register budget for 2 resident 512-thread blocks per SM (<= 64 registers; measured fastest)
#endif
//
// Same three passes as above, built from the radix-16 register stages of
// fft16.cuh: G rows (pass A/C) or CC columns (pass B) per block, interleaved
// in padded shared memory; the first and last stages read and write global
// memory (or registers) directly, and pass B multiplies by Lambda between its
// forward and inverse column transforms without leaving registers.

template <typename T, int G>
__global__ void __launch_bounds__(512, KRY_K16_MINB) k16_pass_a(const T* __restrict__ vin, int64_t ld, const double* __restrict__ scale,
                                                  int nvec, int pair0, const int* __restrict__ rowptr,
                                                  const int* __restrict__ colidx, int n1, int n2, int M2, int C,
                                                  int logC, int PS, typename cx_of<T>::type* __restrict__ slab,
                                                  const void* tw32, const void* tw64, const int* __restrict__ skip) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    const int L = M2, b = 31 - __clz(L), LT = L >> 4;
    const int g = threadIdx.x % G, t = threadIdx.x / G;
    const int row = blockIdx.x * G + g;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;
    if (skip && skip[va] && (!has_b || skip[vb])) return;   // both columns finished (whole block)
    const Cx* tw = twiddles<T>(tw32, tw64);
    const Cx zero = cmk<Cx>((T)0, (T)0);

    for (int pos = t; pos < n2; pos += LT) buf[kry16::spos(pos, PS, G, g)] = zero;
    __syncthreads();
    if (row < n1) {
        const T sa = scale ? (T)scale[va] : (T)1;
        const T sb = (scale && has_b) ? (T)scale[vb] : (T)1;
        const T* pa = vin + (int64_t)va * ld;
        const T* pb = vin + (int64_t)vb * ld;
        const int q1 = rowptr[row + 1];
        for (int q = rowptr[row] + t; q < q1; q += LT)
            buf[kry16::spos(colidx[q], PS, G, g)] = cmk<Cx>(pa[q] * sa, has_b ? pb[q] * sb : (T)0);
    }
    __syncthreads();

    Cx* out = slab + (int64_t)blockIdx.y * n1 * M2 + (int64_t)row * C;
    const int64_t tstride = (int64_t)n1 * C;
    auto ld_s = [&](int pos) { return buf[kry16::spos(pos, PS, G, g)]; };
    auto ld_0 = [&](int pos) { return pos < n2 ? buf[kry16::spos(pos, PS, G, g)] : zero; };
    auto st_s = [&](int pos, Cx z) { buf[kry16::spos(pos, PS, G, g)] = z; };
    auto st_g = [&](int pos, Cx z) {
        if (row < n1) out[(int64_t)(pos >> logC) * tstride + (pos & (C - 1))] = z;
    };
    Cx v[16];
    kry16::transform<Cx, false, true>(b, v, t, tw, ld_0, ld_s, st_s, st_g, true, false);
}

template <typename T, int CC>
__global__ void __launch_bounds__(512, KRY_K16_MINB) k16_pass_b(typename cx_of<T>::type* __restrict__ slab,
                                                  const T* __restrict__ lamT, int n1, int M1, int M2, int PS,
                                                  const void* tw32, const void* tw64, int pair0, int64_t lam_stride,
                                                  int vpt, const int* __restrict__ skip, int nvec) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    if (skip) {
        const int va = 2 * (pair0 + (int)blockIdx.y), vb = va + 1;
        if (skip[va] && (vb >= nvec || skip[vb])) return;
    }
    const int L = M1, b = 31 - __clz(L), LT = L >> 4;
    const int c = threadIdx.x % CC, t = threadIdx.x / CC;
    const int tile = blockIdx.x;
    Cx* blk = slab + (int64_t)blockIdx.y * n1 * M2 + (int64_t)tile * n1 * CC;
    const Cx* tw = twiddles<T>(tw32, tw64);
    const Cx zero = cmk<Cx>((T)0, (T)0);

    auto ld_g = [&](int pos) { return pos < n1 ? blk[pos * CC + c] : zero; };
    auto ld_s = [&](int pos) { return buf[kry16::spos(pos, PS, CC, c)]; };
    auto st_s = [&](int pos, Cx z) { buf[kry16::spos(pos, PS, CC, c)] = z; };
    auto st_g = [&](int pos, Cx z) {
        if (pos < n1) blk[pos * CC + c] = z;
    };
    const int nst = kry16::num_stages(b);
    Cx v[16];
    // forward column transform, ending in registers (slot m = row t + m L/16)
    {
        const int r0 = kry16::stage_radix(b, 0);
        // rows >= n1 (>= M1/2) are zero: half-input first stage
        using LDG = decltype(ld_g)&;
        using STS = decltype(st_s)&;
        switch (r0) {
            case 2: kry16::stage<Cx, 2, false, LDG, STS, true>(v, t, L, 1, tw, ld_g, st_s, false); break;
            case 4: kry16::stage<Cx, 4, false, LDG, STS, true>(v, t, L, 1, tw, ld_g, st_s, false); break;
            case 8: kry16::stage<Cx, 8, false, LDG, STS, true>(v, t, L, 1, tw, ld_g, st_s, false); break;
            default: kry16::stage<Cx, 16, false, LDG, STS, true>(v, t, L, 1, tw, ld_g, st_s, false); break;
        }
        __syncthreads();
        int Ns = r0;
#pragma unroll 1
        for (int s = 1; s < nst - 1; ++s) {
            kry16::stage<Cx, 16, false>(v, t, L, Ns, tw, ld_s, st_s, true);
            __syncthreads();
            Ns *= 16;
        }
        kry16::last_stage_regs<Cx, false>(v, t, L, Ns, tw, ld_s, true);
    }
    // eigenvalue multiply (scaled by 1/(M1 M2))
    const int theta = vpt ? (2 * (pair0 + (int)blockIdx.y)) / vpt : 0;
    const T* lam = lamT + theta * lam_stride + (int64_t)(tile * CC + c) * L;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const T l = lam[t + m * LT];
        v[m] = cmk<Cx>(v[m].x * l, v[m].y * l);
    }
    // inverse column transform, starting from registers, keeping rows < n1
    {
        const int r0 = kry16::stage_radix(b, 0);
        kry16::first_stage_regs<Cx, true>(r0, v, t, L, tw, st_s);
        __syncthreads();
        int Ns = r0;
#pragma unroll 1
        for (int s = 1; s < nst - 1; ++s) {
            kry16::stage<Cx, 16, true>(v, t, L, Ns, tw, ld_s, st_s, true);
            __syncthreads();
            Ns *= 16;
        }
        kry16::stage<Cx, 16, true>(v, t, L, Ns, tw, ld_s, st_g, false);
    }
}

template <typename T, int G, int MODE>
__global__ void __launch_bounds__(512, KRY_K16_MINB) k16_pass_c(const typename cx_of<T>::type* __restrict__ slab,
                                                  const T* __restrict__ vin, int64_t ld_in,
                                                  const double* __restrict__ scale, T* __restrict__ vout,
                                                  int64_t ld_out, int nvec, int pair0, const int* __restrict__ rowptr,
                                                  const int* __restrict__ colidx, int n1, int n2, int M2, int C,
                                                  int logC, int PS, double tau2, double* __restrict__ dots,
                                                  int ndot_stride, const void* tw32, const void* tw64,
                                                  const double* __restrict__ tau2v, int vpt,
                                                  const int* __restrict__ skip) {
    using Cx = typename cx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Cx* buf = reinterpret_cast<Cx*>(smem_raw);
    __shared__ double red[2][32];
    const int L = M2, b = 31 - __clz(L), LT = L >> 4;
    const int g = threadIdx.x % G, t = threadIdx.x / G;
    const int row = blockIdx.x * G + g;
    const int pair = pair0 + blockIdx.y;
    const int va = 2 * pair, vb = 2 * pair + 1;
    const bool has_b = vb < nvec;
    if (skip && skip[va] && (!has_b || skip[vb])) return;   // both columns finished (whole block)
    const Cx* tw = twiddles<T>(tw32, tw64);
    const Cx zero = cmk<Cx>((T)0, (T)0);

    const Cx* in = slab + (int64_t)blockIdx.y * n1 * M2 + (int64_t)row * C;
    const int64_t tstride = (int64_t)n1 * C;
    auto ld_g = [&](int pos) {
        return row < n1 ? in[(int64_t)(pos >> logC) * tstride + (pos & (C - 1))] : zero;
    };
    auto ld_s = [&](int pos) { return buf[kry16::spos(pos, PS, G, g)]; };
    auto st_s = [&](int pos, Cx z) { buf[kry16::spos(pos, PS, G, g)] = z; };
    auto st_n = [&](int pos, Cx z) {
        if (pos < n2) buf[kry16::spos(pos, PS, G, g)] = z;
    };
    Cx v[16];
    kry16::transform<Cx, true>(b, v, t, tw, ld_g, ld_s, st_s, st_n, false, true);
    __syncthreads();

    DotAcc<T> acc_a, acc_b;
    if (row < n1) {
        if (MODE == 0) {
            const T sa = scale ? (T)scale[va] : (T)1;
            const T sb = (scale && has_b) ? (T)scale[vb] : (T)1;
            const T t2 = (T)(tau2v ? tau2v[vpt ? va / vpt : 0] : tau2);
            const T* pa = vin + (int64_t)va * ld_in;
            const T* pb = vin + (int64_t)vb * ld_in;
            T* oa = vout + (int64_t)va * ld_out;
            T* ob = vout + (int64_t)vb * ld_out;
            const int q1 = rowptr[row + 1];
            for (int q = rowptr[row] + t; q < q1; q += LT) {
                const Cx z = buf[kry16::spos(colidx[q], PS, G, g)];
                const T xa = pa[q] * sa;
                const T ya = z.x + t2 * xa;
                oa[q] = ya;
                acc_a.add_prod(xa, ya);
                if (has_b) {
                    const T xb = pb[q] * sb;
                    const T yb = z.y + t2 * xb;
                    ob[q] = yb;
                    acc_b.add_prod(xb, yb);
                }
            }
        } else {
            T* oa = vout + (int64_t)va * ld_out + (int64_t)row * n2;
            T* ob = vout + (int64_t)vb * ld_out + (int64_t)row * n2;
            for (int j = t; j < n2; j += LT) {
                const Cx z = buf[kry16::spos(j, PS, G, g)];
                oa[j] = z.x;
                if (has_b) ob[j] = z.y;
            }
        }
    }
    if (MODE == 0 && dots != nullptr) {
        double da = acc_a.value(), db = acc_b.value();
        // rows are interleaved across lanes (g fastest); the block reduction
        // sums every row's products of the block in a fixed order
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
            double sa = 0.0, sb = 0.0;
            const int nw = (blockDim.x >= 32) ? (blockDim.x >> 5) : blockDim.x;
            for (int k = 0; k < nw; ++k) {
                sa += red[0][k];
                sb += red[1][k];
            }
            dots[(int64_t)va * ndot_stride + blockIdx.x] = sa;
            if (has_b) dots[(int64_t)vb * ndot_stride + blockIdx.x] = sb;
        }
    }
}

// ------------------------------------------------------------------ host side

static size_t cx_size(bool dbl) { return dbl ? sizeof(double2) : sizeof(float2); }

int smem_limit(kry_ctx* ctx) { return ctx->max_smem_optin; }

template <typename T>
struct MvLaunch {
    using Cx = typename cx_of<T>::type;

    template <int EPT, int G>
    static void a(dim3 grid, int threads, size_t smem, cudaStream_t s, const T* vin, int64_t ld, const double* scale,
                  int nvec, int pair0, const int* rowptr, const int* colidx, int n1, int M2, int C, Cx* slab,
                  const void* tw32, const void* tw64) {
        auto k = k_pass_a<T, EPT, G>;
        KRY_ALLOW_MAX_SMEM(k);
        k<<<grid, threads, smem, s>>>(vin, ld, scale, nvec, pair0, rowptr, colidx, n1, M2, C, slab, tw32, tw64);
        KRY_CHECK_LAUNCH();
    }
    template <int EPT, int CC>
    static void b(dim3 grid, int threads, size_t smem, cudaStream_t s, Cx* slab, const T* lamT, int n1, int M1, int M2,
                  const void* tw32, const void* tw64, int pair0 = 0, int64_t lam_stride = 0, int vpt = 0) {
        auto k = k_pass_b<T, EPT, CC>;
        KRY_ALLOW_MAX_SMEM(k);
        k<<<grid, threads, smem, s>>>(slab, lamT, n1, M1, M2, tw32, tw64, pair0, lam_stride, vpt);
        KRY_CHECK_LAUNCH();
    }
    template <int EPT, int G, int MODE>
    static void c(dim3 grid, int threads, size_t smem, cudaStream_t s, const Cx* slab, const T* vin, int64_t ld_in,
                  const double* scale, T* vout, int64_t ld_out, int nvec, int pair0, const int* rowptr,
                  const int* colidx, int n1, int n2, int M2, int C, double tau2, double* dots, int nds,
                  const void* tw32, const void* tw64, const double* tau2v = nullptr, int vpt = 0) {
        auto k = k_pass_c<T, EPT, G, MODE>;
        KRY_ALLOW_MAX_SMEM(k);
        k<<<grid, threads, smem, s>>>(slab, vin, ld_in, scale, vout, ld_out, nvec, pair0, rowptr, colidx, n1, n2, M2,
                                      C, tau2, dots, nds, tw32, tw64, tau2v, vpt);
        KRY_CHECK_LAUNCH();
    }
};

#define KRY_DISPATCH_EG(EPTV, GV, CALL)                                               \
    do {                                                                              \
        if (EPTV == 8) {                                                              \
            if (GV == 1) { constexpr int E_ = 8, G_ = 1; CALL; }                       \
            else if (GV == 2) { constexpr int E_ = 8, G_ = 2; CALL; }                  \
            else if (GV == 4) { constexpr int E_ = 8, G_ = 4; CALL; }                  \
            else if (GV == 8) { constexpr int E_ = 8, G_ = 8; CALL; }                  \
            else throw KryError{KRY_EUNSUPPORTED, "bad group count"};                \
        } else if (EPTV == 16) {                                                      \
            if (GV == 1) { constexpr int E_ = 16, G_ = 1; CALL; }                      \
            else if (GV == 2) { constexpr int E_ = 16, G_ = 2; CALL; }                 \
            else if (GV == 4) { constexpr int E_ = 16, G_ = 4; CALL; }                 \
            else if (GV == 8) { constexpr int E_ = 16, G_ = 8; CALL; }                 \
            else throw KryError{KRY_EUNSUPPORTED, "bad group count"};                \
        } else                                                                        \
            throw KryError{KRY_EUNSUPPORTED, "bad elements per thread"};              \
    } while (0)

// Pick a schedule that fits shared memory and the 1024-thread block limit.
static MvSched pick_sched(kry_ctx* ctx, const MvSched& want, int M1, int M2, bool dbl) {
    MvSched s = want;
    const size_t cs = cx_size(dbl);
    const size_t lim = (size_t)ctx->max_smem_optin - 1024;   // leave room for static shared memory
    auto fix = [&](int& ept, int& grp, int L) {
        if (ept != 8 && ept != 16) ept = 8;
        if (L < ept) ept = 8;
        if (L / ept > 1024) ept = 16;
        const int maxthr = (ept >= 16) ? 512 : 1024;
        while (grp > 1 && ((size_t)grp * (L + 1) * cs > lim || grp * (L / ept) > maxthr)) grp /= 2;
    };
    fix(s.ept_row, s.rows_per_cta, M2);
    fix(s.ept_col, s.cols_per_cta, M1);
    return s;
}

// ---- radix-16 path: schedule, shared-memory pad shift and launches

#ifndef KRY_SMEM_CARVEOUT
#define KRY_SMEM_CARVEOUT -1   // L1 / shared-memory split: driver default (measured fastest)
#endif

void prof_record(kry_ctx* ctx, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    KRY_CUDA(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        KRY_CUDA(cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal));
    else
        KRY_CUDA(cudaEventRecord(ev, ctx->stream));
}

static bool use16(int M1, int M2) { return M1 >= 64 && M2 >= 64 && M1 <= KRY_MAX_M && M2 <= KRY_MAX_M; }

// Pad shift of the interleaved shared-memory layout for NT transforms of
// length L (chosen from a bank-conflict model of the stage access patterns).
static int pad_shift(int L, int NT) {
    if (L >= 4096) return 4;
    if (L == 2048) return NT == 1 ? 4 : 3;
    if (NT >= 4) return 2;
    if (NT == 2) return 3;
    return 4;
}

static size_t smem16(int L, int NT, bool dbl) {
    return (size_t)(L + (L >> pad_shift(L, NT))) * NT * cx_size(dbl);
}

static int ilog2(int x) { return 31 - __builtin_clz((unsigned)x); }

static int batch_bucket(int nvec) {
    int b = 1;
    while (b < nvec && b < 64) b <<= 1;
    return b;
}

uint64_t sched_key(int M1, int M2, bool dbl, int nvec) {
    return (uint64_t)M1 | ((uint64_t)M2 << 16) | ((uint64_t)(dbl ? 1 : 0) << 32) | ((uint64_t)batch_bucket(nvec) << 40);
}

const MvSched& sched_for(kry_ctx* ctx, int M1, int M2, bool dbl, int nvec) {
    auto it = ctx->tuned.find(sched_key(M1, M2, dbl, nvec));
    if (it != ctx->tuned.end()) return it->second;
    return dbl ? ctx->sched64 : ctx->sched32;
}

// Rows per block (pass A/C) and columns per block (pass B, = slab tile width).
static void sched16(kry_ctx* ctx, int M1, int M2, bool dbl, int nvec, int* G, int* C) {
    const MvSched& want = sched_for(ctx, M1, M2, dbl, nvec);
    const size_t lim = (size_t)ctx->max_smem_optin - 1024;   // leave room for static shared memory
    // the length-specialised FP32 passes run up to 8 transforms per block
    const int ntmax = (!dbl && ctx->use_spec) ? 8 : 16;
    auto fit = [&](int L, int nt) {
        nt = std::max(1, std::min(nt, ntmax));
        while (nt > 1 && (nt * (L >> 4) > (ntmax == 8 ? 1024 : 512) || smem16(L, nt, dbl) > lim)) nt >>= 1;
        return nt;
    };
    int g = want.g16 > 0 ? want.g16 : std::max(1, 256 / (M2 >> 4));
    int c = want.c16 > 0 ? want.c16 : std::max(1, 512 / (M1 >> 4));
    *G = fit(M2, g);
    *C = std::min(fit(M1, c), M2);
    if (ntmax == 8) *C = std::min(*C, std::max(1, M2 >> 4));   // specialised pass A/C need C <= M2 / 16
}

#define KRY_DISPATCH_NT(NTV, ...)                                  \
    do {                                                            \
        switch (NTV) {                                              \
            case 1: { constexpr int N_ = 1; __VA_ARGS__; } break;          \
            case 2: { constexpr int N_ = 2; __VA_ARGS__; } break;          \
            case 4: { constexpr int N_ = 4; __VA_ARGS__; } break;          \
            case 8: { constexpr int N_ = 8; __VA_ARGS__; } break;          \
            case 16: { constexpr int N_ = 16; __VA_ARGS__; } break;        \
            default: throw KryError{KRY_EUNSUPPORTED, "bad transforms per block"}; \
        }                                                           \
    } while (0)

template <typename T>
static void run_matvec16(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
                         int64_t ld_out, int nvec, double tau2, double* dots, int nds, int mode,
                         typename cx_of<T>::type* slab, int ppb, int vpt, const int* skip) {
    const bool dbl = sizeof(T) == 8;
    const int n1 = e->n1, n2 = e->n2, M1 = e->M1, M2 = e->M2;
    int G, C;
    sched16(ctx, M1, M2, dbl, nvec, &G, &C);
    const int npairs = (nvec + 1) / 2;
    const T* lamT = dbl ? reinterpret_cast<const T*>(e->lam64T) : reinterpret_cast<const T*>(e->lam32T);
    const int* rowptr = ctx->rowptr.as<int>();
    const int* colidx = ctx->colidx.as<int>();
    const void* tw32 = ctx->tw32.p;
    const void* tw64 = ctx->tw64.p;
    cudaStream_t st = ctx->stream;
    const int psA = pad_shift(M2, G), psB = pad_shift(M1, C);
    const int thrA = G * (M2 >> 4), thrB = C * (M1 >> 4);
    const size_t smA = smem16(M2, G, dbl), smB = smem16(M1, C, dbl);
    const int nbx = (n1 + G - 1) / G;
    const int logC = ilog2(C);
    if constexpr (sizeof(T) == 4) {
        if (mode == 0 && ctx->use_spec && kspec::supported(M1, M2, G, C)) {
            kspec::SpecArgs a{};
            a.vin = vin; a.ld_in = ld_in; a.scale = scale; a.vout = vout; a.ld_out = ld_out;
            a.nvec = nvec; a.rowptr = rowptr; a.colidx = colidx;
            a.n1 = n1; a.n2 = n2; a.M1 = M1; a.M2 = M2; a.G = G; a.C = C; a.logC = logC;
            KRY_REQUIRE(e->lam32P != nullptr, KRY_EINVAL, "embedding lacks the permuted eigenvalues");
            a.slab = slab; a.lamP = e->lam32P; a.lam_stride = e->lam_stride; a.vpt = vpt;
            a.tau2 = tau2; a.tau2v = ctx->no_nugget ? nullptr : e->tau2_dev; a.dots = dots; a.nds = nds;
            a.twt = ctx->twt32.as<float4>(); a.skip = skip;
            for (int pair0 = 0; pair0 < npairs; pair0 += ppb) {
                a.pair0 = pair0;
                a.np = std::min(ppb, npairs - pair0);
                KRY_REQUIRE(kspec::launch_a(a, st) && kspec::launch_b(a, st) && kspec::launch_c(a, st),
                            KRY_EUNSUPPORTED, "no specialised matvec pass for this shape");
            }
            return;
        }
    }
    for (int pair0 = 0; pair0 < npairs; pair0 += ppb) {
        const int np = std::min(ppb, npairs - pair0);
        dim3 gA(nbx, np), gB(M2 / C, np);
        KRY_DISPATCH_NT(G, {
            auto k = k16_pass_a<T, N_>;
            KRY_ALLOW_MAX_SMEM(k);
            KRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, KRY_SMEM_CARVEOUT));
            k<<<gA, thrA, smA, st>>>(vin, ld_in, scale, nvec, pair0, rowptr, colidx, n1, n2, M2, C, logC, psA, slab,
                                    tw32, tw64, skip);
            KRY_CHECK_LAUNCH();
        });
        KRY_DISPATCH_NT(C, {
            auto k = k16_pass_b<T, N_>;
            KRY_ALLOW_MAX_SMEM(k);
            KRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, KRY_SMEM_CARVEOUT));
            k<<<gB, thrB, smB, st>>>(slab, lamT, n1, M1, M2, psB, tw32, tw64, pair0, e->lam_stride, vpt, skip, nvec);
            KRY_CHECK_LAUNCH();
        });
        if (mode == 0) {
            KRY_DISPATCH_NT(G, {
                auto k = k16_pass_c<T, N_, 0>;
                KRY_ALLOW_MAX_SMEM(k);
                KRY_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, KRY_SMEM_CARVEOUT));
                k<<<gA, thrA, smA, st>>>(slab, vin, ld_in, scale, vout, ld_out, nvec, pair0, rowptr, colidx, n1, n2,
                                        M2, C, logC, psA, tau2, dots, nds, tw32, tw64, ctx->no_nugget ? nullptr : e->tau2_dev, vpt, skip);
                KRY_CHECK_LAUNCH();
            });
        } else {
            KRY_DISPATCH_NT(G, {
                auto k = k16_pass_c<T, N_, 1>;
                KRY_ALLOW_MAX_SMEM(k);
                k<<<gA, thrA, smA, st>>>(slab, vin, ld_in, scale, vout, ld_out, nvec, pair0, rowptr, colidx, n1, n2,
                                        M2, C, logC, psA, tau2, dots, nds, tw32, tw64, ctx->no_nugget ? nullptr : e->tau2_dev, vpt, skip);
                KRY_CHECK_LAUNCH();
            });
        }
    }
}

template <typename T>
static void run_matvec(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
                       int64_t ld_out, int nvec, double tau2, double* dots, int nds, int mode, int vpt = 0,
                       const int* skip = nullptr);

// Irregular sites (sites.cu): A^T by scatter onto the whole grid, sigma^2 Sigma
// on the whole grid by the FFT passes with whole-grid index lists and no
// nugget, then (mode 0) the gather A, nugget and dot partials; in mode 1 the
// whole-grid result is the output.
template <typename T>
static void run_matvec_sites(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale,
                             T* vout, int64_t ld_out, int nvec, double tau2, double* dots, int nds, int mode, int vpt,
                             const int* skip) {
    const int64_t N = (int64_t)e->n1 * e->n2;
    KRY_REQUIRE(ctx->rowptr_full.p && ctx->full_n1 == e->n1 && ctx->full_n2 == e->n2, KRY_EINVAL,
                "the site map's whole-grid index lists are missing");
    DevBuf& gb = sizeof(T) == 8 ? ctx->sites.grid64 : ctx->sites.grid32;
    gb.ensure((size_t)(mode == 0 ? 2 : 1) * nvec * N * sizeof(T));
    T* gin = gb.as<T>();
    T* gout = (mode == 0) ? gin + (size_t)nvec * N : vout;
    site_scatter<T>(ctx, vin, ld_in, scale, nvec, gin, skip);
    struct Scope {   // whole-grid lists in, the site map and the nugget out, for the FFT passes
        kry_ctx* c;
        int64_t p;
        explicit Scope(kry_ctx* x) : c(x), p(x->p) {
            std::swap(c->rowptr, c->rowptr_full);
            std::swap(c->colidx, c->colidx_full);
            c->p = (int64_t)c->n1 * c->n2;
            c->sites.active = false;
            c->no_nugget = true;
        }
        ~Scope() {
            std::swap(c->rowptr, c->rowptr_full);
            std::swap(c->colidx, c->colidx_full);
            c->p = p;
            c->sites.active = true;
            c->no_nugget = false;
        }
    } scope(ctx);
    run_matvec<T>(ctx, e, gin, N, nullptr, gout, mode == 0 ? N : ld_out, nvec, 0.0, nullptr, 0, 0, vpt, skip);
    if (mode == 0) {
        ctx->p = scope.p;   // the gather runs over the sites
        ctx->sites.active = true;
        site_gather<T>(ctx, gout, vin, ld_in, scale, vout, ld_out, nvec, tau2, e->tau2_dev, vpt, dots, nds, skip);
    }
}

template <typename T>
static void run_matvec(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
                       int64_t ld_out, int nvec, double tau2, double* dots, int nds, int mode, int vpt,
                       const int* skip) {
    KRY_REQUIRE(vpt == 0 || (vpt % 2 == 0 && nvec % vpt == 0 && nvec / vpt <= e->ntheta), KRY_EINVAL,
                "vectors per theta must be even and divide the batch");
    if (ctx->sites.active) {
        run_matvec_sites<T>(ctx, e, vin, ld_in, scale, vout, ld_out, nvec, tau2, dots, nds, mode, vpt, skip);
        return;
    }
    using Cx = typename cx_of<T>::type;
    const bool dbl = sizeof(T) == 8;
    const int n1 = e->n1, n2 = e->n2, M1 = e->M1, M2 = e->M2;
    if (use16(M1, M2)) {
        const int npairs = (nvec + 1) / 2;
        const MvSched& want = sched_for(ctx, M1, M2, dbl, nvec);
        const int ppb = want.pairs_per_batch > 0 ? std::min(want.pairs_per_batch, npairs) : npairs;
        DevBuf& sb = dbl ? ctx->slab64 : ctx->slab32;
        sb.ensure((size_t)n1 * M2 * cx_size(dbl) * ppb);
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (ctx->prof_on) {
            KRY_CUDA(cudaEventCreate(&ev0));
            KRY_CUDA(cudaEventCreate(&ev1));
            prof_record(ctx, ev0);
        }
        run_matvec16<T>(ctx, e, vin, ld_in, scale, vout, ld_out, nvec, tau2, dots, nds, mode, sb.as<Cx>(), ppb, vpt,
                        skip);
        if (ctx->prof_on) {
            prof_record(ctx, ev1);
            ctx->prof_ev.push_back(ev0);
            ctx->prof_ev.push_back(ev1);
            ctx->prof_nvec.push_back(nvec);
            ctx->prof_dbl.push_back(dbl ? 1 : 0);
        }
        return;
    }
    MvSched s = pick_sched(ctx, dbl ? ctx->sched64 : ctx->sched32, M1, M2, dbl);
    const int npairs = (nvec + 1) / 2;
    int ppb = s.pairs_per_batch > 0 ? std::min(s.pairs_per_batch, npairs) : npairs;
    const size_t slab_pair = (size_t)n1 * M2 * cx_size(dbl);
    DevBuf& sb = dbl ? ctx->slab64 : ctx->slab32;
    sb.ensure(slab_pair * ppb);
    Cx* slab = sb.as<Cx>();
    const T* lamT = dbl ? reinterpret_cast<const T*>(e->lam64T) : reinterpret_cast<const T*>(e->lam32T);
    const int C = s.cols_per_cta;
    const int G = s.rows_per_cta;
    const int* rowptr = ctx->rowptr.as<int>();
    const int* colidx = ctx->colidx.as<int>();
    const void* tw32 = ctx->tw32.p;
    const void* tw64 = ctx->tw64.p;
    cudaStream_t st = ctx->stream;
    const int thrA = G * (M2 / s.ept_row);
    const size_t smA = (size_t)G * (M2 + 1) * cx_size(dbl);
    const int thrB = C * (M1 / s.ept_col);
    const size_t smB = (size_t)C * (M1 + 1) * cx_size(dbl);
    const int nbx = (n1 + G - 1) / G;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (ctx->prof_on) {
        KRY_CUDA(cudaEventCreate(&ev0));
        KRY_CUDA(cudaEventCreate(&ev1));
        prof_record(ctx, ev0);
    }
    for (int pair0 = 0; pair0 < npairs; pair0 += ppb) {
        const int np = std::min(ppb, npairs - pair0);
        dim3 gA(nbx, np), gB(M2 / C, np);
        KRY_DISPATCH_EG(s.ept_row, G,
                        (MvLaunch<T>::template a<E_, G_>(gA, thrA, smA, st, vin, ld_in, scale, nvec, pair0, rowptr,
                                                         colidx, n1, M2, C, slab, tw32, tw64)));
        KRY_DISPATCH_EG(s.ept_col, C,
                        (MvLaunch<T>::template b<E_, G_>(gB, thrB, smB, st, slab, lamT, n1, M1, M2, tw32, tw64, pair0,
                                                         e->lam_stride, vpt)));
        if (mode == 0) {
            KRY_DISPATCH_EG(s.ept_row, G,
                            (MvLaunch<T>::template c<E_, G_, 0>(gA, thrA, smA, st, slab, vin, ld_in, scale, vout,
                                                                ld_out, nvec, pair0, rowptr, colidx, n1, n2, M2, C,
                                                                tau2, dots, nds, tw32, tw64, ctx->no_nugget ? nullptr : e->tau2_dev, vpt)));
        } else {
            KRY_DISPATCH_EG(s.ept_row, G,
                            (MvLaunch<T>::template c<E_, G_, 1>(gA, thrA, smA, st, slab, vin, ld_in, scale, vout,
                                                                ld_out, nvec, pair0, rowptr, colidx, n1, n2, M2, C,
                                                                tau2, dots, nds, tw32, tw64, ctx->no_nugget ? nullptr : e->tau2_dev, vpt)));
        }
    }
    if (ctx->prof_on) {
        prof_record(ctx, ev1);
        ctx->prof_ev.push_back(ev0);
        ctx->prof_ev.push_back(ev1);
        ctx->prof_nvec.push_back(nvec);
        ctx->prof_dbl.push_back(dbl ? 1 : 0);
    }
}

// Number of per-block dot partials pass C writes per vector for a batch of
// nvec vectors (the Krylov finalisers sum exactly this many).
int matvec_num_partials(kry_ctx* ctx, const kry_embed* e, bool dbl, int nvec) {
    if (ctx->sites.active) return site_num_partials(ctx);
    if (use16(e->M1, e->M2)) {
        int G, C;
        sched16(ctx, e->M1, e->M2, dbl, nvec, &G, &C);
        return (e->n1 + G - 1) / G;
    }
    MvSched s = pick_sched(ctx, dbl ? ctx->sched64 : ctx->sched32, e->M1, e->M2, dbl);
    return (e->n1 + s.rows_per_cta - 1) / s.rows_per_cta;
}

template <typename T>
void matvec_ex(kry_ctx* ctx, const kry_embed* e, const T* vin, int64_t ld_in, const double* scale, T* vout,
               int64_t ld_out, int nvec, double* dots, int nds, int vpt, const int* skip) {
    run_matvec<T>(ctx, e, vin, ld_in, scale, vout, ld_out, nvec, e->cov.tau2, dots, nds, 0, vpt, skip);
}

template void matvec_ex<float>(kry_ctx*, const kry_embed*, const float*, int64_t, const double*, float*, int64_t, int,
                               double*, int, int, const int*);
template void matvec_ex<double>(kry_ctx*, const kry_embed*, const double*, int64_t, const double*, double*, int64_t,
                                int, double*, int, int, const int*);

template <typename T>
void matvec(kry_ctx* ctx, const kry_embed* e, const T* vin, T* vout, int nvec, int64_t ld, double) {
    run_matvec<T>(ctx, e, vin, ld, nullptr, vout, ld, nvec, e->cov.tau2, nullptr, 0, 0);
}
template void matvec<float>(kry_ctx*, const kry_embed*, const float*, float*, int, int64_t, double);
template void matvec<double>(kry_ctx*, const kry_embed*, const double*, double*, int, int64_t, double);

void sigma_to_grid64(kry_ctx* ctx, const kry_embed* e, const double* vin, double* out_grid, int nvec, int64_t ld,
                     int vpt) {
    run_matvec<double>(ctx, e, vin, ld, nullptr, out_grid, (int64_t)e->n1 * e->n2, nvec, 0.0, nullptr, 0, 1, vpt);
}

// ------------------------------------------------------------------ allocation-free matvec
//
// kry_matvec_noalloc serves callers that cannot allocate device memory when
// they call: applications whose device memory is all owned by their own pool
// or arena (a framework's caching allocator that has reserved the GPU), and
// latency-critical loops that cannot absorb the device-wide synchronisation of
// cudaMalloc / cudaFree.  It runs the same FFT passes as kry_matvec, chosen by
// the same schedule, but its slab lives in a fixed file-scope device array
// instead of context scratch, taking as many complex pairs per batch as the
// array holds.  The array is part of the module, so every GPU that loads this
// library holds it until the process exits.
//
// Set-up: the first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it with the
// identity of the device's current CUDA context; a later call under another
// context (after cudaDeviceReset, say) looks it up again.  Make that first call
// before any stream capture.  The context, its mask and the embedding must
// already exist (creating them does allocate).
//
// Sharing: every call on a device uses the same array and it keeps the last
// call's contents.  Nothing needs clearing, because pass A writes every slab
// element that passes B and C read.  Calls whose work overlaps on the GPU
// (other streams, other host threads) race on the array and must be
// serialised by the caller.

#define KRY_NOALLOC_SCRATCH_BYTES (16u << 20)   // 16 MiB: one 1024 x 1024 FP32 complex pair
#define KRY_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[KRY_NOALLOC_SCRATCH_BYTES];

struct NoallocSlot {
    void* addr = nullptr;
    unsigned long long ctx_id = 0;
};
static std::mutex g_noalloc_mu;
static NoallocSlot g_noalloc_slot[KRY_NOALLOC_MAX_DEVICES];

// Identity of the calling thread's current CUDA context (driver entry points
// cuCtxGetCurrent / cuCtxGetId, looked up through the runtime), 0 if unknown.
static unsigned long long current_ctx_id() {
    typedef int (*GetCurrentFn)(void**);
    typedef int (*GetIdFn)(void*, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // under g_noalloc_mu
        looked_up = true;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrentFn>(f1);
            get_id = reinterpret_cast<GetIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    void* c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != 0 || c == nullptr || get_id(c, &id) != 0) return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device (looked up once
// per device and context).
static void* noalloc_scratch(int device) {
    KRY_REQUIRE(device >= 0 && device < KRY_NOALLOC_MAX_DEVICES, KRY_EUNSUPPORTED,
                "device index too large for the allocation-free matvec");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot& slot = g_noalloc_slot[device];
    const unsigned long long id = current_ctx_id();
    if (slot.addr == nullptr || slot.ctx_id != id) {
        void* ptr = nullptr;
        cudaError_t err = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (err != cudaSuccess)
            throw KryError{KRY_ECUDA, std::string("cudaGetSymbolAddress of the static matvec scratch failed: ") +
                                          cudaGetErrorString(err)};
        slot.addr = ptr;
        slot.ctx_id = id;
    }
    return slot.addr;
}

template <typename T>
static void run_matvec_noalloc(kry_ctx* ctx, const kry_embed* e, const T* vin, T* vout, int nvec, int64_t ld,
                               void* scratch) {
    using Cx = typename cx_of<T>::type;
    const bool dbl = sizeof(T) == 8;
    const int n1 = e->n1, n2 = e->n2, M1 = e->M1, M2 = e->M2;
    const size_t slab_pair = (size_t)n1 * M2 * cx_size(dbl);
    KRY_REQUIRE(slab_pair <= KRY_NOALLOC_SCRATCH_BYTES, KRY_EUNSUPPORTED,
                "grid too large for the allocation-free matvec: n1 * M2 * sizeof(complex) = " +
                    std::to_string(slab_pair) + " bytes exceeds its 16 MiB static scratch");
    const int npairs = (nvec + 1) / 2;
    const int cap = std::max(1, (int)(KRY_NOALLOC_SCRATCH_BYTES / slab_pair));
    Cx* slab = static_cast<Cx*>(scratch);
    const double tau2 = e->cov.tau2;
    if (use16(M1, M2)) {
        // the passes and schedule of kry_matvec, with at most `cap` pairs per batch
        const MvSched& want = sched_for(ctx, M1, M2, dbl, nvec);
        int ppb = want.pairs_per_batch > 0 ? std::min(want.pairs_per_batch, npairs) : npairs;
        ppb = std::min(ppb, cap);
        run_matvec16<T>(ctx, e, vin, ld, nullptr, vout, ld, nvec, tau2, nullptr, 0, 0, slab, ppb, 0, nullptr);
        return;
    }
    // transform lengths below 64: the generic radix-8 passes, as kry_matvec
    MvSched s = pick_sched(ctx, dbl ? ctx->sched64 : ctx->sched32, M1, M2, dbl);
    int ppb = s.pairs_per_batch > 0 ? std::min(s.pairs_per_batch, npairs) : npairs;
    ppb = std::min(ppb, cap);
    const T* lamT = dbl ? reinterpret_cast<const T*>(e->lam64T) : reinterpret_cast<const T*>(e->lam32T);
    const int C = s.cols_per_cta;
    const int G = s.rows_per_cta;
    const int* rowptr = ctx->rowptr.as<int>();
    const int* colidx = ctx->colidx.as<int>();
    const void* tw32 = ctx->tw32.p;
    const void* tw64 = ctx->tw64.p;
    cudaStream_t st = ctx->stream;
    const int thrA = G * (M2 / s.ept_row);
    const size_t smA = (size_t)G * (M2 + 1) * cx_size(dbl);
    const int thrB = C * (M1 / s.ept_col);
    const size_t smB = (size_t)C * (M1 + 1) * cx_size(dbl);
    const int nbx = (n1 + G - 1) / G;
    for (int pair0 = 0; pair0 < npairs; pair0 += ppb) {
        const int np = std::min(ppb, npairs - pair0);
        dim3 gA(nbx, np), gB(M2 / C, np);
        KRY_DISPATCH_EG(s.ept_row, G,
                        (MvLaunch<T>::template a<E_, G_>(gA, thrA, smA, st, vin, ld, nullptr, nvec, pair0, rowptr,
                                                         colidx, n1, M2, C, slab, tw32, tw64)));
        KRY_DISPATCH_EG(s.ept_col, C,
                        (MvLaunch<T>::template b<E_, G_>(gB, thrB, smB, st, slab, lamT, n1, M1, M2, tw32, tw64, pair0,
                                                         e->lam_stride, 0)));
        KRY_DISPATCH_EG(s.ept_row, G,
                        (MvLaunch<T>::template c<E_, G_, 0>(gA, thrA, smA, st, slab, vin, ld, nullptr, vout, ld,
                                                            nvec, pair0, rowptr, colidx, n1, n2, M2, C, tau2,
                                                            nullptr, 0, tw32, tw64, e->tau2_dev, 0)));
    }
}

}  // namespace kry

extern "C" kry_status kry_matvec_noalloc(kry_ctx* ctx, const kry_embed* e, const void* v_dev, void* out_dev,
                                         int32_t nvec, int64_t ld) {
    if (!ctx) return KRY_EINVAL;
    try {
        KRY_CUDA(cudaSetDevice(ctx->device));
        ctx->err.clear();
        KRY_REQUIRE(e != nullptr && e->ctx == ctx, KRY_EINVAL, "embedding is NULL or belongs to another context");
        KRY_REQUIRE(ctx->p > 0 && e->n1 == ctx->n1 && e->n2 == ctx->n2, KRY_EINVAL,
                    "no mask set, or the embedding grid differs from the mask grid");
        KRY_REQUIRE(!ctx->sites.active, KRY_EUNSUPPORTED,
                    "the allocation-free matvec needs an observation mask (kry_set_mask), not sites");
        KRY_REQUIRE(nvec >= 0 && ld >= ctx->p, KRY_EINVAL, "need nvec >= 0 and ld >= p");
        if (nvec == 0) return KRY_OK;
        KRY_REQUIRE(v_dev && out_dev, KRY_EINVAL, "v_dev and out_dev must not be NULL");
        void* scratch = kry::noalloc_scratch(ctx->device);
        if (e->prec == KRY_F64)
            kry::run_matvec_noalloc<double>(ctx, e, static_cast<const double*>(v_dev), static_cast<double*>(out_dev),
                                            nvec, ld, scratch);
        else
            kry::run_matvec_noalloc<float>(ctx, e, static_cast<const float*>(v_dev), static_cast<float*>(out_dev),
                                           nvec, ld, scratch);
        return KRY_OK;
    } catch (const KryError& err) {
        ctx->err = err.msg;
        return err.st;
    } catch (const std::exception& err) {
        ctx->err = err.what();
        return KRY_ECUDA;
    }
}

// ------------------------------------------------------------------ schedule autotuner
//
// Times every feasible radix-16 schedule (rows per block for the row passes,
// columns per block = slab tile width for the column pass, complex pairs per
// batch: all at once, or chunks whose slab stays within ~32 or ~64 MB of L2)
// on the caller's embedding and batch width, and caches the fastest for
// (M1, M2, precision, batch bucket).

namespace kry {

template <typename T>
__global__ void k_fill_test(T* __restrict__ x, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (T)(((i * 2654435761ll) & 1023) - 511) * (T)(1.0 / 512.0);
}

template <typename T>
static double time_sched(kry_ctx* ctx, const kry_embed* e, const T* v, T* out, int nvec, int reps) {
    cudaEvent_t a, b;
    KRY_CUDA(cudaEventCreate(&a));
    KRY_CUDA(cudaEventCreate(&b));
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;
    run_matvec<T>(ctx, e, v, ctx->p, nullptr, out, ctx->p, nvec, e->cov.tau2, nullptr, 0, 0);   // warm-up
    KRY_CUDA(cudaEventRecord(a, ctx->stream));
    for (int r = 0; r < reps; ++r)
        run_matvec<T>(ctx, e, v, ctx->p, nullptr, out, ctx->p, nvec, e->cov.tau2, nullptr, 0, 0);
    KRY_CUDA(cudaEventRecord(b, ctx->stream));
    KRY_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    KRY_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->prof_on = prof;
    return ms / reps;
}

template <typename T>
static double autotune_t(kry_ctx* ctx, const kry_embed* e, int nvec, MvSched* best_out) {
    const bool dbl = sizeof(T) == 8;
    const int M1 = e->M1, M2 = e->M2;
    const uint64_t key = sched_key(M1, M2, dbl, nvec);
    const size_t n = (size_t)nvec * ctx->p;
    DevBuf tv, to;
    tv.stream = to.stream = ctx->stream;
    tv.ensure(n * sizeof(T));
    to.ensure(n * sizeof(T));
    k_fill_test<T><<<1024, 256, 0, ctx->stream>>>(tv.as<T>(), (int64_t)n);
    KRY_CHECK_LAUNCH();
    const int npairs = (nvec + 1) / 2;
    const size_t slab_pair = (size_t)e->n1 * M2 * cx_size(dbl);
    std::vector<int> ppbs = {0};
    for (size_t budget : {(size_t)32 << 20, (size_t)64 << 20}) {
        const int c = (int)std::max<size_t>(1, budget / slab_pair);
        if (c < npairs && std::find(ppbs.begin(), ppbs.end(), c) == ppbs.end()) ppbs.push_back(c);
    }
    const size_t lim = (size_t)ctx->max_smem_optin - 1024;   // leave room for static shared memory
    double best = 1e30;
    MvSched bs = dbl ? ctx->sched64 : ctx->sched32;
    const bool had = ctx->tuned.count(key) > 0;
    const MvSched prev = had ? ctx->tuned[key] : bs;
    if (use16(M1, M2)) {
        const bool spec = !dbl && ctx->use_spec;
        const int tmax = spec ? 1024 : 512;
        for (int g : {1, 2, 4, 8, 16}) {
            if (g * (M2 >> 4) > tmax || smem16(M2, g, dbl) > lim || (spec && g > 8)) continue;
            for (int c : {1, 2, 4, 8, 16}) {
                if (c * (M1 >> 4) > tmax || smem16(M1, c, dbl) > lim || c > M2 || (spec && (c > 8 || c > (M2 >> 4)))) continue;
                for (int ppb : ppbs) {
                    MvSched cand = bs;
                    cand.g16 = g;
                    cand.c16 = c;
                    cand.pairs_per_batch = ppb;
                    ctx->tuned[key] = cand;
                    const double ms = time_sched<T>(ctx, e, tv.as<T>(), to.as<T>(), nvec, 3);
                    if (ms < best) {
                        best = ms;
                        bs = cand;
                    }
                }
            }
        }
        ctx->tuned[key] = bs;
    } else {
        if (had) ctx->tuned[key] = prev;
        best = time_sched<T>(ctx, e, tv.as<T>(), to.as<T>(), nvec, 3);
    }
    tv.release();
    to.release();
    if (best_out) *best_out = bs;
    return best;
}

double autotune(kry_ctx* ctx, const kry_embed* e, int nvec, MvSched* best) {
    return e->prec == KRY_F64 ? autotune_t<double>(ctx, e, nvec, best) : autotune_t<float>(ctx, e, nvec, best);
}

}  // namespace kry

extern "C" kry_status kry_autotune(kry_ctx* ctx, const kry_embed* e, int32_t nvec, double* best_ms,
                                   int32_t* rows_per_block, int32_t* cols_per_block, int32_t* pairs_per_batch) {
    if (!ctx) return KRY_EINVAL;
    try {
        KRY_CUDA(cudaSetDevice(ctx->device));
        ctx->err.clear();
        KRY_REQUIRE(e != nullptr && e->ctx == ctx, KRY_EINVAL, "embedding is NULL or belongs to another context");
        KRY_REQUIRE(ctx->p > 0 && e->n1 == ctx->n1 && e->n2 == ctx->n2, KRY_EINVAL,
                    "no mask set, or the embedding grid differs from the mask grid");
        KRY_REQUIRE(nvec >= 1, KRY_EINVAL, "nvec must be >= 1");
        MvSched b;
        const double ms = kry::autotune(ctx, e, nvec, &b);
        if (best_ms) *best_ms = ms;
        if (rows_per_block) *rows_per_block = b.g16;
        if (cols_per_block) *cols_per_block = b.c16;
        if (pairs_per_batch) *pairs_per_batch = b.pairs_per_batch;
        return KRY_OK;
    } catch (const KryError& err) {
        ctx->err = err.msg;
        return err.st;
    } catch (const std::exception& err) {
        ctx->err = err.what();
        return KRY_ECUDA;
    }
}

extern "C" kry_status kry_set_schedule(kry_ctx* ctx, const kry_embed* e, int32_t nvec, int32_t rows_per_block,
                                       int32_t cols_per_block, int32_t pairs_per_batch) {
    if (!ctx) return KRY_EINVAL;
    try {
        KRY_REQUIRE(e != nullptr && e->ctx == ctx, KRY_EINVAL, "embedding is NULL or belongs to another context");
        auto pow2 = [](int x) { return x >= 0 && (x & (x - 1)) == 0; };
        KRY_REQUIRE(nvec >= 1 && pow2(rows_per_block) && pow2(cols_per_block) && rows_per_block <= 16 &&
                        cols_per_block <= 16 && pairs_per_batch >= 0,
                    KRY_EINVAL, "rows/cols per block must be 0 (default) or a power of two <= 16; pairs >= 0");
        const bool dbl = e->prec == KRY_F64;
        MvSched s = dbl ? ctx->sched64 : ctx->sched32;
        s.g16 = rows_per_block;
        s.c16 = cols_per_block;
        s.pairs_per_batch = pairs_per_batch;
        ctx->tuned[kry::sched_key(e->M1, e->M2, dbl, nvec)] = s;
        return KRY_OK;
    } catch (const KryError& err) {
        ctx->err = err.msg;
        return err.st;
    }
}
