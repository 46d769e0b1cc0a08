// Irregular observation sites (Sec. 2): y = X beta + A x + eps with the latent
// field x on the n1 x n2 grid and A the p x n mapping matrix of Wendland
// weights.  Row i of A holds, for the cell centres c_j within one grid
// spacing of site s_i along both axes,
//   A_ij = w(d_ij) / sum_k w(d_ik),  w(d) = (1 - d)^4_+ (1 + 4 d),
//   d_ij = max(|s_i1 - c_j1| / dx1, |s_i2 - c_j2| / dx2),
// so at most the 2 x 2 centres around a site carry weight; near the border of
// the domain only the centres that exist are normalised over (a site inside
// the domain always has a centre within half a spacing on both axes).
//
// The covariance matvec K v = sigma^2 A Sigma A^T v + tau^2 v then runs as
//   1. scatter A^T v onto the whole grid (k_site_scatter: per cell, the sum of
//      its entries in site order, so the result does not depend on scheduling);
//   2. sigma^2 Sigma on the whole grid by the circulant-embedding FFT passes
//      (the observed-cell passes with whole-grid index lists and no nugget);
//   3. gather A (k_site_gather: four weights per site), add the nugget and
//      form the per-block dot-product partials the Krylov loops consume.
// Steps 1 and 3 are defined here; matvec.cu sequences the three.
#include <math.h>

#include <algorithm>

#include "kry_internal.cuh"

namespace kry {

namespace {

unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

__device__ __forceinline__ double wendland_w(double d) {
    if (!(d < 1.0)) return 0.0;
    const double a = 1.0 - d;
    const double a2 = a * a;
    return a2 * a2 * (1.0 + 4.0 * d);
}

// Per site: the cells of its 2 x 2 neighbourhood of centres (-1 where the
// weight is zero or the centre lies outside the grid), the normalised
// weights, and the entry count of each cell.  A site outside the domain
// [0, n1 dx1] x [0, n2 dx2] (or not finite) sets *bad and gets no entry.
__global__ void k_site_weights(const double* __restrict__ sites, int64_t p, int n1, int n2, double dx1, double dx2,
                               int* __restrict__ corner, double* __restrict__ w64, float* __restrict__ w32,
                               int* __restrict__ cnt, int* __restrict__ bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        const double s1 = sites[2 * i], s2 = sites[2 * i + 1];
        const bool inside = s1 >= 0.0 && s1 <= n1 * dx1 && s2 >= 0.0 && s2 <= n2 * dx2;
        double w[4] = {0.0, 0.0, 0.0, 0.0};
        int c[4] = {-1, -1, -1, -1};
        double tot = 0.0;
        if (inside) {
            const double u1 = s1 / dx1 - 0.5, u2 = s2 / dx2 - 0.5;   // site in cell-centre index units
            const int b1 = (int)floor(u1), b2 = (int)floor(u2);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j1 = b1 + (k >> 1), j2 = b2 + (k & 1);
                if (j1 < 0 || j1 >= n1 || j2 < 0 || j2 >= n2) continue;
                const double d = fmax(fabs(u1 - j1), fabs(u2 - j2));
                w[k] = wendland_w(d);
                if (w[k] > 0.0) c[k] = j1 * n2 + j2;
                tot += w[k];
            }
        }
        if (!(tot > 0.0)) {
            atomicOr(bad, 1);
            tot = 1.0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double a = (c[k] >= 0) ? w[k] / tot : 0.0;
            corner[4 * i + k] = c[k];
            w64[4 * i + k] = a;
            w32[4 * i + k] = (float)a;
            if (c[k] >= 0) atomicAdd(&cnt[c[k]], 1);
        }
    }
}

// Entry count of each grid row (one block per row).
__global__ void k_row_totals(const int* __restrict__ cnt, int n2, int* __restrict__ rowtot) {
    const int row = blockIdx.x;
    int s = 0;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) s += cnt[(int64_t)row * n2 + j];
    __shared__ int red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        rowtot[row] = t;
    }
}

// Exclusive scan of the row totals (one thread; n1 <= 4096): rowbase[n1] = total.
__global__ void k_row_bases(const int* __restrict__ rowtot, int n1, int* __restrict__ rowbase) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < n1; ++i) {
            rowbase[i] = s;
            s += rowtot[i];
        }
        rowbase[n1] = s;
    }
}

// cellptr[c] = first entry of cell c: the row's base plus the exclusive scan of
// the counts within the row (one block of 256 threads per row, each thread a
// contiguous chunk of cells).  cellptr[N] = total.
__global__ void k_cell_ptr(const int* __restrict__ cnt, const int* __restrict__ rowbase, int n1, int n2,
                           int* __restrict__ cellptr) {
    const int row = blockIdx.x;
    const int per = (n2 + blockDim.x - 1) / blockDim.x;
    const int j0 = threadIdx.x * per, j1 = min(n2, j0 + per);
    const int64_t base = (int64_t)row * n2;
    int s = 0;
    for (int j = j0; j < j1; ++j) s += cnt[base + j];
    __shared__ int pre[256];
    pre[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = rowbase[row];
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int v = pre[t];
            pre[t] = acc;
            acc += v;
        }
    }
    __syncthreads();
    int acc = pre[threadIdx.x];
    for (int j = j0; j < j1; ++j) {
        cellptr[base + j] = acc;
        acc += cnt[base + j];
    }
    if (row == n1 - 1 && threadIdx.x == 0) cellptr[(int64_t)n1 * n2] = rowbase[n1];
}

// Entries of A^T grouped by cell (cursor: zeroed counts).
__global__ void k_site_fill(const int* __restrict__ corner, const double* __restrict__ w64, int64_t p,
                            const int* __restrict__ cellptr, int* __restrict__ cursor, int* __restrict__ ent_site,
                            double* __restrict__ ent_w64) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = corner[4 * i + k];
            if (c < 0) continue;
            const int pos = cellptr[c] + atomicAdd(&cursor[c], 1);
            ent_site[pos] = (int)i;
            ent_w64[pos] = w64[4 * i + k];
        }
}

// Sort each cell's entries by site (insertion sort: a cell has few entries),
// so the scatter sums in a fixed order; then the FP32 copy of the weights.
__global__ void k_cell_sort(const int* __restrict__ cellptr, int64_t N, int* __restrict__ ent_site,
                            double* __restrict__ ent_w64, float* __restrict__ ent_w32) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int a = cellptr[c], b = cellptr[c + 1];
        for (int i = a + 1; i < b; ++i) {
            const int s = ent_site[i];
            const double w = ent_w64[i];
            int j = i - 1;
            while (j >= a && ent_site[j] > s) {
                ent_site[j + 1] = ent_site[j];
                ent_w64[j + 1] = ent_w64[j];
                --j;
            }
            ent_site[j + 1] = s;
            ent_w64[j + 1] = w;
        }
        for (int i = a; i < b; ++i) ent_w32[i] = (float)ent_w64[i];
    }
}

__global__ void k_full_lists(int* __restrict__ rowptr, int* __restrict__ colidx, int n1, int n2) {
    const int64_t N = (int64_t)n1 * n2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        colidx[i] = (int)(i % n2);
        if (i % n2 == 0) rowptr[i / n2] = (int)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rowptr[n1] = (int)N;
}

// Step 1: grid[v][c] = scale[v] * sum over the entries of cell c of w * vin[v][site].
template <typename T>
__global__ void k_site_scatter(const int* __restrict__ cellptr, const int* __restrict__ ent_site,
                               const T* __restrict__ ent_w, const T* __restrict__ vin, int64_t ld_in,
                               const double* __restrict__ scale, int64_t N, T* __restrict__ grid,
                               const int* __restrict__ skip) {
    const int v = blockIdx.y;
    // skipped as the FFT passes skip: only when both columns of the complex
    // pair are (a skipped column's grid still enters its partner's transform,
    // and rounding there depends on it)
    const int w = v ^ 1;
    if (skip && skip[v] && (w >= (int)gridDim.y || skip[w])) return;
    const T s = scale ? (T)scale[v] : (T)1;
    const T* x = vin + (int64_t)v * ld_in;
    T* g = grid + (int64_t)v * N;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (int64_t)gridDim.x * blockDim.x) {
        const int a = cellptr[c], b = cellptr[c + 1];
        T acc = (T)0;
        for (int e = a; e < b; ++e) acc += ent_w[e] * x[ent_site[e]];
        g[c] = acc * s;
    }
}

// Step 3: vout[v][i] = sum_k w_ik grid[v][cell_ik] + tau2 x_i with x = scale[v] vin[v];
// per-block partials of x^T vout (fixed-order block reduction, one slot per block).
template <typename T>
__global__ void k_site_gather(const int* __restrict__ corner, const T* __restrict__ w, const T* __restrict__ grid,
                              int64_t N, const T* __restrict__ vin, int64_t ld_in, const double* __restrict__ scale,
                              T* __restrict__ vout, int64_t ld_out, int64_t p, double tau2,
                              const double* __restrict__ tau2v, int vpt, double* __restrict__ dots, int nds,
                              const int* __restrict__ skip) {
    const int v = blockIdx.y;
    if (skip && skip[v]) return;
    const T s = scale ? (T)scale[v] : (T)1;
    const T t2 = (T)(tau2v ? tau2v[vpt ? v / vpt : 0] : tau2);
    const T* x = vin + (int64_t)v * ld_in;
    const T* g = grid + (int64_t)v * N;
    T* y = vout + (int64_t)v * ld_out;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += (int64_t)gridDim.x * blockDim.x) {
        T z = (T)0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = corner[4 * i + k];
            if (c >= 0) z += w[4 * i + k] * g[c];
        }
        const T xi = x[i] * s;
        const T yi = z + t2 * xi;
        y[i] = yi;
        acc += (double)xi * (double)yi;
    }
    if (dots == nullptr) return;
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        dots[(int64_t)v * nds + blockIdx.x] = t;
    }
}

}  // namespace

// Blocks (and dot partials per vector) of the site gather.
int site_num_partials(kry_ctx* ctx) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(256, (ctx->p + 255) / 256));
}

template <typename T>
void site_scatter(kry_ctx* ctx, const T* vin, int64_t ld_in, const double* scale, int nvec, T* grid,
                  const int* skip) {
    const int64_t N = (int64_t)ctx->n1 * ctx->n2;
    const bool dbl = sizeof(T) == 8;
    const T* w = dbl ? reinterpret_cast<const T*>(ctx->sites.ent_w64.p) : reinterpret_cast<const T*>(ctx->sites.ent_w32.p);
    dim3 g(grid_for(N), nvec);
    k_site_scatter<T><<<g, 256, 0, ctx->stream>>>(ctx->sites.cellptr.as<int>(), ctx->sites.ent_site.as<int>(), w, vin,
                                                  ld_in, scale, N, grid, skip);
    KRY_CHECK_LAUNCH();
}

template <typename T>
void site_gather(kry_ctx* ctx, const T* grid, const T* vin, int64_t ld_in, const double* scale, T* vout,
                 int64_t ld_out, int nvec, double tau2, const double* tau2v, int vpt, double* dots, int nds,
                 const int* skip) {
    const int64_t N = (int64_t)ctx->n1 * ctx->n2;
    const bool dbl = sizeof(T) == 8;
    const T* w = dbl ? reinterpret_cast<const T*>(ctx->sites.w64.p) : reinterpret_cast<const T*>(ctx->sites.w32.p);
    const int nb = dots ? nds : site_num_partials(ctx);
    dim3 g(nb, nvec);
    k_site_gather<T><<<g, 256, 0, ctx->stream>>>(ctx->sites.corner.as<int>(), w, grid, N, vin, ld_in, scale, vout,
                                                 ld_out, ctx->p, tau2, tau2v, vpt, dots, nds, skip);
    KRY_CHECK_LAUNCH();
}

template void site_scatter<float>(kry_ctx*, const float*, int64_t, const double*, int, float*, const int*);
template void site_scatter<double>(kry_ctx*, const double*, int64_t, const double*, int, double*, const int*);
template void site_gather<float>(kry_ctx*, const float*, const float*, int64_t, const double*, float*, int64_t, int,
                                 double, const double*, int, double*, int, const int*);
template void site_gather<double>(kry_ctx*, const double*, const double*, int64_t, const double*, double*, int64_t,
                                  int, double, const double*, int, double*, int, const int*);

// Build the site structures of ctx for nsite sites (device coordinates,
// row-major pairs) on the grid's cells; returns false if a site lies outside
// the domain.
bool build_sites(kry_ctx* ctx, int n1, int n2, double dx1, double dx2, const double* sites, int64_t nsite) {
    cudaStream_t st = ctx->stream;
    const int64_t N = (int64_t)n1 * n2;
    auto& S = ctx->sites;
    S.corner.ensure((size_t)4 * nsite * sizeof(int));
    S.w64.ensure((size_t)4 * nsite * sizeof(double));
    S.w32.ensure((size_t)4 * nsite * sizeof(float));
    S.cellptr.ensure((size_t)(N + 1) * sizeof(int));
    S.cnt.ensure((size_t)(N + n1 + (n1 + 1) + 1) * sizeof(int));
    int* cnt = S.cnt.as<int>();
    int* rowtot = cnt + N;
    int* rowbase = rowtot + n1;
    int* bad = rowbase + (n1 + 1);
    KRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(N + n1 + (n1 + 1) + 1) * sizeof(int), st));
    k_site_weights<<<grid_for(nsite), 256, 0, st>>>(sites, nsite, n1, n2, dx1, dx2, S.corner.as<int>(),
                                                    S.w64.as<double>(), S.w32.as<float>(), cnt, bad);
    KRY_CHECK_LAUNCH();
    k_row_totals<<<n1, 256, 0, st>>>(cnt, n2, rowtot);
    KRY_CHECK_LAUNCH();
    k_row_bases<<<1, 32, 0, st>>>(rowtot, n1, rowbase);
    KRY_CHECK_LAUNCH();
    k_cell_ptr<<<n1, 256, 0, st>>>(cnt, rowbase, n1, n2, S.cellptr.as<int>());
    KRY_CHECK_LAUNCH();
    int* hp = reinterpret_cast<int*>(ctx->host_pinned);
    KRY_CUDA(cudaMemcpyAsync(hp, rowbase + n1, sizeof(int), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaMemcpyAsync(hp + 1, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    KRY_CUDA(cudaStreamSynchronize(st));
    const int64_t nnz = hp[0];
    if (hp[1]) return false;
    S.ent_site.ensure((size_t)std::max<int64_t>(1, nnz) * sizeof(int));
    S.ent_w64.ensure((size_t)std::max<int64_t>(1, nnz) * sizeof(double));
    S.ent_w32.ensure((size_t)std::max<int64_t>(1, nnz) * sizeof(float));
    KRY_CUDA(cudaMemsetAsync(cnt, 0, (size_t)N * sizeof(int), st));
    k_site_fill<<<grid_for(nsite), 256, 0, st>>>(S.corner.as<int>(), S.w64.as<double>(), nsite, S.cellptr.as<int>(),
                                                 cnt, S.ent_site.as<int>(), S.ent_w64.as<double>());
    KRY_CHECK_LAUNCH();
    k_cell_sort<<<grid_for(N), 256, 0, st>>>(S.cellptr.as<int>(), N, S.ent_site.as<int>(), S.ent_w64.as<double>(),
                                             S.ent_w32.as<float>());
    KRY_CHECK_LAUNCH();
    // whole-grid index lists of the FFT passes (step 2)
    ctx->rowptr_full.ensure((size_t)(n1 + 1) * sizeof(int));
    ctx->colidx_full.ensure((size_t)N * sizeof(int));
    k_full_lists<<<grid_for(N), 256, 0, st>>>(ctx->rowptr_full.as<int>(), ctx->colidx_full.as<int>(), n1, n2);
    KRY_CHECK_LAUNCH();
    ctx->full_n1 = n1;
    ctx->full_n2 = n2;
    KRY_CUDA(cudaStreamSynchronize(st));
    return true;
}

}  // namespace kry
