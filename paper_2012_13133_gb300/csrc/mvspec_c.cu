// Pass C of the specialised FP32 matvec (mvspec.cuh) for every supported
// (log2 M2, rows per block).
#include "kry_internal.cuh"
#include "mvspec.cuh"

namespace kspec {

namespace {
struct RunC {
    const SpecArgs& a;
    cudaStream_t st;
    template <int B, int NT>
    bool run() const {
        auto k = ks_pass_c<B, NT>;
        KRY_ALLOW_MAX_SMEM(k);
        dim3 grid((a.n1 + NT - 1) / NT, a.np);
        launch_pdl(k, grid, dim3(tpb(B, NT)), smem_bytes(B, NT), st, a.slab, a.vin, a.ld_in, a.scale, a.vout, a.ld_out, a.nvec,
                                                       a.pair0, a.rowptr, a.colidx, a.n1, a.n2, a.C, a.logC, a.tau2,
                                                       a.dots, a.nds, a.twt, a.tau2v, a.vpt, a.skip);
        return true;
    }
};
}  // namespace

bool launch_c(const SpecArgs& a, cudaStream_t st) { return dispatch(ilog2i(a.M2), a.G, RunC{a, st}); }

}  // namespace kspec
