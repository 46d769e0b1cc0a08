// genGK / genHyBR (Sec. 3.2, Alg. 1; Eq. prof_lik) with the options of
// kry_genhybr_prec: prec KRY_F32 keeps the Krylov vectors and the whole-grid
// matvec in FP32 (FP64 scalars and reductions); reorth reorthogonalises each
// new u against U (Euclidean) and each new v against V (Sigma inner product),
// two Gram-Schmidt passes.  Arguments otherwise as kry::genhybr.
#pragma once

#include "kry_internal.cuh"

namespace kry {

void genhybr_opt(kry_ctx* ctx, const kry_cov& cov, kry_prec prec, bool reorth, const double* b, int k, double* x_out,
                 double* alphas, double* betas, double* z2, double* psi2, double* pl, double* grad, double* psi_out);

}  // namespace kry
