// Pass A of the specialised FP32 matvec (mvspec.cuh) for every supported
// (log2 M2, rows per block), the shape check and the stage twiddle table.
#include "kry_internal.cuh"
#include "mvspec.cuh"

namespace kspec {

bool supported(int M1, int M2, int G, int C) {
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    if (!pow2(M1) || !pow2(M2) || M1 < 64 || M2 < 64 || M1 > 8192 || M2 > 8192) return false;
    if (!pow2(G) || !pow2(C) || G > 8 || C > 8 || C > (M2 >> 4)) return false;
    return G * (M2 >> 4) <= 1024 && C * (M1 >> 4) <= 1024;
}

__global__ void k_stage_twiddles(float2* __restrict__ twt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TWT_ROWS * 16) return;
    const int row = i >> 4, m = i & 15;
    const int ns = 1 << (31 - __clz(row + 1));   // row = ns - 1 + k, k < ns
    const int k = row + 1 - ns;
    double s, c;
    sincospi(-2.0 * (double)(k * m) / (16.0 * (double)ns), &s, &c);
    twt[i] = make_float2((float)c, (float)s);
}

void fill_stage_twiddles(float2* twt_dev, cudaStream_t st) {
    k_stage_twiddles<<<(TWT_ROWS * 16 + 255) / 256, 256, 0, st>>>(twt_dev);
    KRY_CHECK_LAUNCH();
}

namespace {
struct RunA {
    const SpecArgs& a;
    cudaStream_t st;
    template <int B, int NT>
    bool run() const {
        auto k = ks_pass_a<B, NT>;
        KRY_ALLOW_MAX_SMEM(k);
        dim3 grid((a.n1 + NT - 1) / NT, a.np);
        launch_pdl(k, grid, dim3(tpb(B, NT)), smem_bytes(B, NT), st, a.vin, a.ld_in, a.scale, a.nvec, a.pair0,
                   a.rowptr, a.colidx, a.n1, a.n2, a.C, a.logC, a.slab, a.twt, a.skip);
        return true;
    }
};
}  // namespace

bool launch_a(const SpecArgs& a, cudaStream_t st) { return dispatch(ilog2i(a.M2), a.G, RunA{a, st}); }

}  // namespace kspec
