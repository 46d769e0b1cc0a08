// Double-float arithmetic (an unevaluated FP32 pair hi + lo) for the FP32 path.
//
// GB300's FP64 pipe runs at a small fraction of its FP32 rate, so per-element
// FP64 work in the FP32 kernels (a float->double conversion and an FP64 FMA per
// product) makes them FP64-bound.  The accumulations below keep FP64-class
// accuracy with FP32 instructions only:
//   * the exact product a*b = p + e, p = fl(a*b), e = fma(a, b, -p) (the FMA
//     computes a*b - p exactly because that difference is representable);
//   * the exact sum a + b = s + t by Knuth's TwoSum (TAOCP vol. 2, 4.2.2).
// The intrinsics round explicitly, so the compiler cannot contract the steps
// into FMAs, which would break the error-free identities.
#pragma once

#include <cuda_runtime.h>

namespace kry {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Running sum of products held as hi + lo; value() converts once to FP64.
struct DFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float s, t;
        two_sum(hi, p, s, t);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(t, e));
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Dot-product accumulator of the vector precision: double-float for FP32
// vectors, plain FP64 FMAs for FP64 vectors.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<float> {
    DFAcc a;
    __device__ __forceinline__ void add_prod(float x, float y) { a.add_prod(x, y); }
    __device__ __forceinline__ double value() const { return a.value(); }
};
template <>
struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double value() const { return s; }
};

// (hi, lo) += (ahi + alo) * p, where ahi + alo is an FP64 coefficient split
// into two floats: the product ahi * p exactly (p1 + e1), alo * p rounded (it
// is 2^-24 of the first), TwoSum into hi, then TwoSum again to renormalise
// (hi and the correction can cancel, so FastTwoSum's ordering may not hold).
__device__ __forceinline__ void df_axpy(float& hi, float& lo, float ahi, float alo, float p) {
    const float p1 = __fmul_rn(ahi, p);
    const float e1 = __fmaf_rn(ahi, p, -p1);
    float s, t;
    two_sum(hi, p1, s, t);
    const float l = __fadd_rn(lo, __fadd_rn(t, __fmaf_rn(alo, p, e1)));
    two_sum(s, l, hi, lo);
}

// Split an FP64 value into hi + lo floats (hi = fl32(a), lo = fl32(a - hi)).
__device__ __forceinline__ void df_split(double a, float& hi, float& lo) {
    hi = (float)a;
    lo = (float)(a - (double)hi);
}

}  // namespace kry
