// Matern correlation in FP64 on the device (Sec. 2):
//   rho_nu(r) = 2^(1-nu) / Gamma(nu) * x^nu K_nu(x),  x = sqrt(2 nu) r,  r = d / range.
//
// nu = 1/2, 3/2, 5/2 use the elementary closed forms (half-integer Bessel
// functions).  Other nu evaluate K_nu(x) from its integral representation
// K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9) by the
// trapezoidal rule, which converges exponentially for this analytic, even,
// double-exponentially decaying integrand (Trefethen & Weideman, "The
// exponentially convergent trapezoidal rule", SIAM Review 2014).  Every term
// is positive, so there is no cancellation.  The step h = min(0.2, 0.5 /
// sqrt(hypot(x, nu))) keeps the discretisation error below ~1e-14 relative
// for nu <= 8 (the strip-of-analyticity bound with the integrand's peak
// curvature ~hypot(x, nu)); summation stops past the integrand's peak
// (sinh t = nu / x) once a term falls below 1e-18 of the sum.
#pragma once

#include <cuda_runtime.h>

__device__ __forceinline__ double kry_besselk_trap(double nu, double x) {
    const double h = fmin(0.2, 0.5 / sqrt(hypot(x, nu)));
    const double tpk = (nu > 0.0) ? asinh(nu / x) : 0.0;
    double s = 0.5 * exp(-x);
    for (int k = 1; k < 4000; ++k) {
        const double t = k * h;
        const double term = exp(-x * cosh(t)) * cosh(nu * t);
        s += term;
        if (t > tpk && term < 1e-18 * s) break;
    }
    return h * s;
}

__device__ __forceinline__ double kry_matern(double r, double nu) {
    const double x = sqrt(2.0 * nu) * r;
    if (nu == 0.5) return exp(-x);
    if (nu == 1.5) return (1.0 + x) * exp(-x);
    if (nu == 2.5) return (1.0 + x + x * x * (1.0 / 3.0)) * exp(-x);
    if (x <= 0.0) return 1.0;
    if (x > 745.0) return 0.0;
    // 2^(1-nu) / Gamma(nu) * x^nu, formed in logs to avoid overflow
    const double lpre = (1.0 - nu) * 0.69314718055994530942 - lgamma(nu) + nu * log(x);
    return exp(lpre) * kry_besselk_trap(nu, x);
}

// d rho_nu / dr (Sec. 2).  Closed forms for nu = 1/2, 3/2, 5/2; otherwise
// d/dx [x^nu K_nu(x)] = -x^nu K_{nu-1}(x) (DLMF 10.29.4) with K_{nu-1} = K_{|nu-1|}
// (K is even in its order), evaluated by the same trapezoidal rule.
__device__ __forceinline__ double kry_matern_dr(double r, double nu) {
    const double s = sqrt(2.0 * nu);
    const double x = s * r;
    if (nu == 0.5) return -exp(-x);
    if (nu == 1.5) return -s * x * exp(-x);
    if (nu == 2.5) return -s * x * (1.0 + x) * exp(-x) * (1.0 / 3.0);
    if (x <= 0.0 || x > 745.0) return 0.0;
    const double lpre = (1.0 - nu) * 0.69314718055994530942 - lgamma(nu) + nu * log(x);
    return -s * exp(lpre) * kry_besselk_trap(fabs(nu - 1.0), x);
}

// Scaled lag d / range under geometric anisotropy: rotate by angle (ca, sa),
// stretch the minor axis by ratio.
__device__ __forceinline__ double kry_scaled_dist(double h1, double h2, double ca, double sa, double ratio,
                                                  double inv_range) {
    const double u = ca * h1 + sa * h2;
    const double v = -sa * h1 + ca * h2;
    return sqrt(u * u + (ratio * v) * (ratio * v)) * inv_range;
}
