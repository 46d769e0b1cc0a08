// Pass B of the specialised FP32 matvec (mvspec.cuh) for every supported
// (log2 M1, columns per block).
#include "kry_internal.cuh"
#include "mvspec.cuh"

namespace kspec {

namespace {
struct RunB {
    const SpecArgs& a;
    cudaStream_t st;
    template <int B, int NT>
    bool run() const {
        auto k = ks_pass_b<B, NT>;
        KRY_ALLOW_MAX_SMEM(k);
        dim3 grid(a.M2 / NT, a.np);
        launch_pdl(k, grid, dim3(tpb(B, NT)), smem_bytes(B, NT), st, a.slab, a.lamP, a.n1, a.M2, a.twt, a.pair0, a.lam_stride,
                                                       a.vpt, a.skip, a.nvec);
        return true;
    }
};
}  // namespace

bool launch_b(const SpecArgs& a, cudaStream_t st) { return dispatch(ilog2i(a.M1), a.C, RunB{a, st}); }

}  // namespace kspec
