// Ensemble products (Section 4.4, Figs. 15-16): every member's running
// maximum depth, the probability that the maximum depth reaches a threshold,
// and percentile maps of the maximum depth over the ensemble.
//
// The running maximum is raised inside the step kernels (march.cuh,
// tma_march.cuh) when tracking is on: 8 more bytes per member-cell-step.
// With particle weights w_i (Eq. 11; equal after a resampling), per cell:
//   P(hmax >= theta) = sum_i w_i [hmax_i >= theta], summed in member order;
//   the a-percentile = the smallest hmax_i with W_i >= a, where
//   W_i = sum over members j with hmax_j <= hmax_i of w_j (member order),
// i.e. the inverse of the weighted empirical distribution function.
#include <algorithm>
#include <vector>

#include "grid.cuh"
#include "tma.cuh"

#define CK FLOOD_CK

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int kCells = 128;     // cells per CTA in the product kernels
constexpr int kMaxLevels = 16;
constexpr int kMaxMembers = 384;  // members staged in shared memory (kCells x 4 B each)

// Resampling moved particle src's state into slot dst: its maximum-depth
// history goes with it.  Grid-stride over (copy, float4).
__global__ void copy_planes_kernel(float* __restrict__ field, const int32_t* __restrict__ n_copy,
                                   const int32_t* __restrict__ dsts, const int32_t* __restrict__ srcs,
                                   size_t plane4)
{
    const int nc = *n_copy;
    const size_t total = (size_t)nc * plane4;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(t / plane4);
        const size_t e = t - (size_t)q * plane4;
        float4* f = reinterpret_cast<float4*>(field);
        f[(size_t)dsts[q] * plane4 + e] = f[(size_t)srcs[q] * plane4 + e];
    }
}

// Start the running maxima at the members' current depths.
__global__ void init_max_kernel(const float* __restrict__ state, const flood::MemberClock* __restrict__ ms,
                                int M, size_t plane, float* __restrict__ field)
{
    const size_t plane4 = plane / 4, total = (size_t)M * plane4;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(t / plane4);
        const size_t e = t - (size_t)m * plane4;
        const float4* h = reinterpret_cast<const float4*>(state + (size_t)(ms[m].cur * M + m) * 3 * plane);
        reinterpret_cast<float4*>(field)[t] = h[e];
    }
}

struct ProdArgs {
    const float* field;   // [M][plane] running maxima
    const double* w;      // [M] particle weights
    int M, ny, nx, ld;
    size_t plane;
    double threshold;
    int n_levels;
    double levels[kMaxLevels];
    float* exceed;        // [ny][nx] (or null)
    float* pct;           // [n_levels][ny][nx] (or null)
};

// One CTA per 128 cells of a row: the members' maxima of those cells are
// staged in shared memory (column per cell, so reads are conflict-free),
// then each thread forms its cell's products.
__global__ void __launch_bounds__(kCells) products_kernel(const ProdArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    double* w = reinterpret_cast<double*>(smem_raw);
    float* v = reinterpret_cast<float*>(w + a.M);  // [M][kCells]
    const int r = blockIdx.y;
    const int c0 = blockIdx.x * kCells;
    const int t = threadIdx.x;
    const int c = c0 + t;
    for (int m = t; m < a.M; m += kCells) w[m] = a.w[m];
    for (int m = 0; m < a.M; ++m)
        v[m * kCells + t] = c < a.nx ? a.field[(size_t)m * a.plane + (size_t)r * a.ld + c] : 0.0f;
    __syncthreads();
    if (c >= a.nx) return;
    const size_t out = (size_t)r * a.nx + c;
    if (a.exceed) {
        double p = 0.0;
        for (int m = 0; m < a.M; ++m)
            if (v[m * kCells + t] >= (float)a.threshold) p += w[m];
        a.exceed[out] = (float)p;
    }
    if (a.pct) {
        float best[kMaxLevels];
        for (int q = 0; q < a.n_levels; ++q) best[q] = __int_as_float(0x7f800000);  // +inf
        for (int i = 0; i < a.M; ++i) {
            const float hi = v[i * kCells + t];
            double W = 0.0;
            for (int j = 0; j < a.M; ++j)
                if (v[j * kCells + t] <= hi) W += w[j];
            for (int q = 0; q < a.n_levels; ++q)
                if (W >= a.levels[q] && hi < best[q]) best[q] = hi;
        }
        // rounding can leave the weights' total just below a level near 1:
        // the largest value then stands for the top of the distribution
        float top = v[t];
        for (int i = 1; i < a.M; ++i) top = fmaxf(top, v[i * kCells + t]);
        for (int q = 0; q < a.n_levels; ++q)
            a.pct[(size_t)q * a.ny * a.nx + out] = best[q] == __int_as_float(0x7f800000) ? top : best[q];
    }
}

size_t products_smem(int M) { return sizeof(double) * M + sizeof(float) * (size_t)M * kCells; }

}  // namespace

namespace flood {

void launch_copy_planes(float* field, const int32_t* n_copy, const int32_t* dsts, const int32_t* srcs,
                        size_t plane, int n_sm, cudaStream_t s)
{
    copy_planes_kernel<<<n_sm * 4, 512, 0, s>>>(field, n_copy, dsts, srcs, plane / 4);
}

}  // namespace flood

extern "C" int flood_track_max_depth(flood_grid* g, int on, void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    cudaStream_t s = S(stream);
    if (!on) {
        CK(g, cudaStreamSynchronize(s));
        g->track_max = false;
        return FLOOD_OK;
    }
    if (!g->hmax_field) {
        int rc = flood::dalloc(g, &g->hmax_field, (size_t)g->M * g->plane);
        if (rc) return rc;
        if (flood::encode_map_3d(&g->hm_map, g->hmax_field, g->ld, g->ny, (uint64_t)g->M,
                                 sizeof(float) * g->ld, sizeof(float) * g->plane, 128, 1, 1) != 0)
            return flood::fail(g, FLOOD_ERR_CUDA, "tensor map of the running maxima");
    }
    init_max_kernel<<<g->n_sm * 4, 512, 0, s>>>(g->state, g->ms + (g->k % 3) * g->M, g->M, g->plane,
                                                g->hmax_field);
    g->launches++;
    CK(g, cudaGetLastError());
    g->track_max = true;
    return FLOOD_OK;
}

extern "C" int flood_get_max_depth(flood_grid* g, int member, float* out, void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->hmax_field || !g->track_max)
        return flood::fail(g, FLOOD_ERR_STATE, "maximum depth is not being tracked");
    if (member < 0 || member >= g->M || !out) return flood::fail(g, FLOOD_ERR_ARG, "bad member or out");
    cudaStream_t s = S(stream);
    CK(g, cudaMemcpy2DAsync(out, sizeof(float) * g->nx, g->hmax_field + (size_t)member * g->plane,
                            sizeof(float) * g->ld, sizeof(float) * g->nx, g->ny, cudaMemcpyDefault, s));
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}

extern "C" int flood_ensemble_products(flood_grid* g, double threshold, int n_levels,
                                       const double* levels, float* exceed, float* pct, void* stream)
{
    const flood::TraceRange range("flood_ensemble_products");
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->hmax_field || !g->track_max)
        return flood::fail(g, FLOOD_ERR_STATE, "maximum depth is not being tracked");
    if (n_levels < 0 || n_levels > kMaxLevels || (n_levels > 0 && (!levels || !pct)))
        return flood::fail(g, FLOOD_ERR_ARG, "need 0 <= n_levels <= 16 with levels and pct");
    if (g->M > kMaxMembers) return flood::fail(g, FLOOD_ERR_ARG, "more than 384 members");
    if (g->ny > 65535) return flood::fail(g, FLOOD_ERR_ARG, "more than 65535 rows");
    ProdArgs a{};
    for (int q = 0; q < n_levels; ++q) {
        if (!(levels[q] > 0.0 && levels[q] <= 1.0))
            return flood::fail(g, FLOOD_ERR_ARG, "levels must lie in (0, 1]");
        a.levels[q] = levels[q];
    }
    cudaStream_t s = S(stream);
    const size_t cells = (size_t)g->ny * g->nx;
    size_t need = (exceed ? cells : 0) + (size_t)n_levels * cells;
    float* buf = nullptr;
    if (need) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(float) * need, s);
        if (e != cudaSuccess)
            return flood::fail(g, e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA,
                               std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    a.field = g->hmax_field;
    a.w = g->w;
    a.M = g->M;
    a.ny = g->ny; a.nx = g->nx; a.ld = g->ld;
    a.plane = g->plane;
    a.threshold = threshold;
    a.n_levels = n_levels;
    a.exceed = exceed ? buf : nullptr;
    a.pct = n_levels ? buf + (exceed ? cells : 0) : nullptr;
    const size_t shm = products_smem(g->M);
    static bool attr = false;
    if (!attr) {
        CK(g, cudaFuncSetAttribute(products_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)products_smem(kMaxMembers)));
        attr = true;
    }
    dim3 grid((g->nx + kCells - 1) / kCells, g->ny);
    products_kernel<<<grid, kCells, shm, s>>>(a);
    g->launches++;
    CK(g, cudaGetLastError());
    if (exceed) CK(g, cudaMemcpyAsync(exceed, a.exceed, sizeof(float) * cells, cudaMemcpyDefault, s));
    if (n_levels)
        CK(g, cudaMemcpyAsync(pct, a.pct, sizeof(float) * cells * n_levels, cudaMemcpyDefault, s));
    if (buf) CK(g, cudaFreeAsync(buf, s));
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}
