// Ensemble products (Section 4.4, Figs. 15-16): every member's running
// maximum depth, the probability that the maximum depth reaches a threshold,
// and percentile maps of the maximum depth over the ensemble.
//
// The running maximum is raised inside the step kernels (march.cuh,
// tma_march.cuh) when tracking is on: 8 more bytes per member-cell-step.
// With particle weights w_i (Eq. 11; equal after a resampling), per cell:
//   P(hmax >= theta) = sum_i w_i [hmax_i >= theta];
//   the a-percentile = the smallest hmax_i with W_i >= a, where
//   W_i = sum over members j with hmax_j <= hmax_i of w_j,
// i.e. the inverse of the weighted empirical distribution function; the sums
// are exact in fixed point (below).
#include <algorithm>
#include <climits>
#include <cmath>
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

// Weighted sums of the products run in fixed point: each weight counts in
// whole units of 2^-60 (rounded to nearest once, on the host), so the sums
// are exact integers and no summation order changes a map.  A level a is
// reached where W * 2^-60 >= a, i.e. W >= A = ceil(a * 2^60); the exceedance
// map is the exact sum scaled by 2^-60, rounded to FP64, then stored as FP32.
constexpr int kLevelsPerPass = 4;

struct ProdArgs {
    const float* field;   // [M][plane] running maxima
    const long long* u;   // [M] weights in units of 2^-60
    int M, ny, nx, ld;
    size_t plane;
    float threshold;
    int n_levels;                  // levels of this pass (<= kLevelsPerPass)
    long long A[kLevelsPerPass];   // level thresholds in units of 2^-60
    int rank[kLevelsPerPass];      // equal weights: 1-based rank reaching the level (M + 1: none)
    long long u_eq;                // equal weights: the common weight
    float* exceed;        // [ny][nx] (or null)
    float* pct;           // [n_levels][ny][nx] of this pass (or null)
};

__device__ __forceinline__ float exceed_value(long long units)
{
    return (float)(__ll2double_rn(units) * 0x1p-60);
}

// Batcher's odd-even merge sort on N (a power of two) slots, every
// comparator ascending (min to the lower slot).  Slots MT..N-1 would hold
// +inf and never move, so every comparator reaching them is left out: the
// network sorts MT slots.  The merge levels (P, K) are template parameters,
// so every slot index is a compile-time constant and the slots stay in
// registers.
template <bool PAIRS, int MT>
__device__ __forceinline__ void compare_exchange(float (&v)[MT], int (&id)[PAIRS ? MT : 1], int i,
                                                 int k)
{
    if (PAIRS) {
        const bool sw = v[i] > v[k];
        const float vi = v[i], vk = v[k];
        const int ii = id[PAIRS ? i : 0], ik = id[PAIRS ? k : 0];
        v[i] = sw ? vk : vi;
        v[k] = sw ? vi : vk;
        id[PAIRS ? i : 0] = sw ? ik : ii;
        id[PAIRS ? k : 0] = sw ? ii : ik;
    } else {
        const float lo = fminf(v[i], v[k]);
        v[k] = fmaxf(v[i], v[k]);
        v[i] = lo;
    }
}

template <bool PAIRS, int N, int MT, int P, int K>
__device__ __forceinline__ void merge_level(float (&v)[MT], int (&id)[PAIRS ? MT : 1])
{
#pragma unroll
    for (int j = K % P; j + K < N; j += 2 * K) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i + j + K < MT && (i + j) / (2 * P) == (i + j + K) / (2 * P))
                compare_exchange<PAIRS, MT>(v, id, i + j, i + j + K);
        }
    }
    if constexpr (K > 1) merge_level<PAIRS, N, MT, P, K / 2>(v, id);
}

template <bool PAIRS, int N, int MT, int P = 1>
__device__ __forceinline__ void odd_even_merge_sort(float (&v)[MT], int (&id)[PAIRS ? MT : 1])
{
    if constexpr (P < N) {
        merge_level<PAIRS, N, MT, P, P>(v, id);
        odd_even_merge_sort<PAIRS, N, MT, 2 * P>(v, id);
    }
}

// v[k] for a run-time k < MT by a tournament on the bits of k (a select per
// pair and level), so that v stays in registers (an indexed read would move
// the whole array to local memory).
template <int MT>
__device__ __forceinline__ float select_slot(const float (&v)[MT], int k)
{
    constexpr int L = MT <= 32 ? 5 : MT <= 64 ? 6 : 7;
    float t[MT];
#pragma unroll
    for (int i = 0; i < MT; ++i) t[i] = v[i];
#pragma unroll
    for (int b = 0; b < L; ++b) {
        const bool hi = (k >> b) & 1;
#pragma unroll
        for (int i = 0; i < ((MT + (1 << b) - 1) >> b); i += 2)
            t[i >> 1] = (((i + 1) << b) < MT && hi) ? t[i + 1] : t[i];
    }
    return t[0];
}

// One thread per cell.  The cell's MT slots (members, then +inf padding)
// are sorted in registers; with equal weights the a-percentile is the
// value of the rank that first reaches a (ranks from the host), otherwise
// the members travel with their values through the sort and one prefix pass
// over their weights finds, per level, the first sorted position whose
// cumulative weight reaches it.  Tied values may come out in any order: the
// first position to reach a level then still holds the tied value.
template <int MT, bool EQUAL>
__global__ void __launch_bounds__(128) sorted_products_kernel(const ProdArgs a)
{
    __shared__ long long us[EQUAL ? 1 : MT];
    if (!EQUAL) {
        for (int j = threadIdx.x; j < MT; j += blockDim.x) us[j] = j < a.M ? a.u[j] : 0;
        __syncthreads();
    }
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= a.nx) return;
    const float* f = a.field + (size_t)r * a.ld + c;
    float v[MT];
    int id[EQUAL ? 1 : MT];
    if (EQUAL) id[0] = 0;
    long long ex = 0;
    int cnt = 0;
    float top = -__int_as_float(0x7f800000);
#pragma unroll
    for (int j = 0; j < MT; ++j) {
        const bool live = j < a.M;
        const float x = live ? __ldcs(f + (size_t)j * a.plane) : __int_as_float(0x7f800000);
        v[j] = x;
        if (!EQUAL) id[EQUAL ? 0 : j] = j;
        if (live) {
            top = fmaxf(top, x);
            if (EQUAL) cnt += x >= a.threshold;
            else if (x >= a.threshold) ex += us[j];
        }
    }
    constexpr int N = MT <= 32 ? 32 : MT <= 64 ? 64 : 128;   // the network's power of two
    odd_even_merge_sort<!EQUAL, N, MT>(v, id);
    const size_t out = (size_t)r * a.nx + c;
    if (a.exceed) a.exceed[out] = exceed_value(EQUAL ? (long long)cnt * a.u_eq : ex);
    if (!a.pct) return;
    int pos[kLevelsPerPass];   // 0-based sorted position holding each level's value (>= M: none)
    if (EQUAL) {
#pragma unroll
        for (int q = 0; q < kLevelsPerPass; ++q) pos[q] = a.rank[q] - 1;
    } else {
#pragma unroll
        for (int q = 0; q < kLevelsPerPass; ++q) pos[q] = 0;
        long long P = 0;
#pragma unroll
        for (int k = 0; k < MT; ++k) {
            P += us[id[EQUAL ? 0 : k]];
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q) pos[q] += P < a.A[q];
        }
    }
#pragma unroll
    for (int q = 0; q < kLevelsPerPass; ++q) {
        if (q >= a.n_levels) break;
        const float sel = select_slot<MT>(v, pos[q]);
        a.pct[(size_t)q * a.ny * a.nx + out] = pos[q] < a.M ? sel : top;
    }
}

// Any member count up to kMaxMembers: the maxima of 128 cells staged in
// shared memory (column per cell, conflict-free), then per cell and member
// i the weight W_i of the members at or below it, an exact integer sum.
__global__ void __launch_bounds__(kCells) staged_products_kernel(const ProdArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    long long* u = reinterpret_cast<long long*>(smem_raw);
    float* v = reinterpret_cast<float*>(u + a.M);  // [M][kCells]
    const int r = blockIdx.y;
    const int c0 = blockIdx.x * kCells;
    const int t = threadIdx.x;
    const int c = c0 + t;
    for (int m = t; m < a.M; m += kCells) u[m] = a.u[m];
    for (int m = 0; m < a.M; ++m)
        v[m * kCells + t] = c < a.nx ? a.field[(size_t)m * a.plane + (size_t)r * a.ld + c] : 0.0f;
    __syncthreads();
    if (c >= a.nx) return;
    const size_t out = (size_t)r * a.nx + c;
    if (a.exceed) {
        long long e = 0;
        for (int m = 0; m < a.M; ++m)
            if (v[m * kCells + t] >= a.threshold) e += u[m];
        a.exceed[out] = exceed_value(e);
    }
    if (a.pct) {
        float best[kLevelsPerPass];
        for (int q = 0; q < kLevelsPerPass; ++q) best[q] = __int_as_float(0x7f800000);  // +inf
        float top = v[t];
        for (int i = 0; i < a.M; ++i) {
            const float hi = v[i * kCells + t];
            top = fmaxf(top, hi);
            long long W = 0;
            for (int j = 0; j < a.M; ++j)
                if (v[j * kCells + t] <= hi) W += u[j];
            for (int q = 0; q < kLevelsPerPass; ++q)
                if (q < a.n_levels && W >= a.A[q] && hi < best[q]) best[q] = hi;
        }
        for (int q = 0; q < a.n_levels; ++q)
            a.pct[(size_t)q * a.ny * a.nx + out] = best[q] == __int_as_float(0x7f800000) ? top : best[q];
    }
}

size_t products_smem(int M) { return sizeof(long long) * M + sizeof(float) * (size_t)M * kCells; }

template <int MT, bool EQUAL>
void launch_sorted(const ProdArgs& a, cudaStream_t s)
{
    dim3 grid((a.nx + 127) / 128, a.ny);
    sorted_products_kernel<MT, EQUAL><<<grid, 128, 0, s>>>(a);
}

// The fastest kernel for the member count and weights: sorted slots in
// registers up to 96 members (128 with equal weights), staged otherwise.
void launch_products(const ProdArgs& a, bool equal, cudaStream_t s)
{
    if (equal && a.M <= 32) launch_sorted<32, true>(a, s);
    else if (equal && a.M <= 64) launch_sorted<64, true>(a, s);
    else if (equal && a.M <= 96) launch_sorted<96, true>(a, s);
    else if (equal && a.M <= 128) launch_sorted<128, true>(a, s);
    else if (!equal && a.M <= 32) launch_sorted<32, false>(a, s);
    else if (!equal && a.M <= 64) launch_sorted<64, false>(a, s);
    else if (!equal && a.M <= 96) launch_sorted<96, false>(a, s);
    else {
        dim3 grid((a.nx + kCells - 1) / kCells, a.ny);
        staged_products_kernel<<<grid, kCells, products_smem(a.M), s>>>(a);
    }
}

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
    long long A[kMaxLevels];
    for (int q = 0; q < n_levels; ++q) {
        if (!(levels[q] > 0.0 && levels[q] <= 1.0))
            return flood::fail(g, FLOOD_ERR_ARG, "levels must lie in (0, 1]");
        A[q] = (long long)std::ceil(std::ldexp(levels[q], 60));   // exact: a * 2^60 <= 2^60
    }
    const int M = g->M;
    cudaStream_t s = S(stream);
    // the weights in whole units of 2^-60, rounded to nearest (ties to even)
    std::vector<double> w(M);
    CK(g, cudaMemcpyAsync(w.data(), g->w, sizeof(double) * M, cudaMemcpyDeviceToHost, s));
    CK(g, cudaStreamSynchronize(s));
    std::vector<long long> u(M);
    long double total = 0.0L;
    for (int m = 0; m < M; ++m) {
        if (!(w[m] >= 0.0 && w[m] <= 1.0))
            return flood::fail(g, FLOOD_ERR_STATE, "particle weights outside [0, 1]");
        u[m] = std::llrint(std::ldexp(w[m], 60));
        total += (long double)u[m];
    }
    if (total >= std::ldexp(1.0L, 62))
        return flood::fail(g, FLOOD_ERR_STATE, "particle weights do not sum to one");
    const bool equal = std::all_of(u.begin(), u.end(), [&](long long x) { return x == u[0]; });
    const size_t cells = (size_t)g->ny * g->nx;
    const size_t need_f = (exceed ? cells : 0) + (size_t)n_levels * cells;
    char* buf = nullptr;
    const size_t bytes = sizeof(long long) * M + sizeof(float) * need_f;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), bytes, s);
    if (e != cudaSuccess)
        return flood::fail(g, e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA,
                           std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    long long* du = reinterpret_cast<long long*>(buf);
    float* dout = reinterpret_cast<float*>(du + M);
    CK(g, cudaMemcpyAsync(du, u.data(), sizeof(long long) * M, cudaMemcpyHostToDevice, s));
    static bool attr = false;
    if (!attr) {
        CK(g, cudaFuncSetAttribute(staged_products_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)products_smem(kMaxMembers)));
        attr = true;
    }
    ProdArgs a{};
    a.field = g->hmax_field;
    a.u = du;
    a.M = M;
    a.ny = g->ny; a.nx = g->nx; a.ld = g->ld;
    a.plane = g->plane;
    a.threshold = (float)threshold;
    a.u_eq = u[0];
    float* pct_dev = dout + (exceed ? cells : 0);
    // one pass per kLevelsPerPass levels (at least one: the exceedance map)
    for (int q0 = 0; q0 == 0 || q0 < n_levels; q0 += kLevelsPerPass) {
        a.n_levels = std::min(kLevelsPerPass, n_levels - q0);
        for (int q = 0; q < kLevelsPerPass; ++q) {
            const bool on = q < a.n_levels;
            a.A[q] = on ? A[q0 + q] : LLONG_MAX;
            // equal weights: the first rank k with k * u >= A (M + 1: no rank reaches it)
            long long k = M + 1;
            if (on && u[0] > 0) k = std::min<long long>(M + 1, (A[q0 + q] + u[0] - 1) / u[0]);
            a.rank[q] = (int)std::max<long long>(k, 1);
        }
        a.exceed = (exceed && q0 == 0) ? dout : nullptr;
        a.pct = a.n_levels > 0 ? pct_dev + (size_t)q0 * cells : nullptr;
        launch_products(a, equal, s);
        g->launches++;
        CK(g, cudaGetLastError());
    }
    if (exceed) CK(g, cudaMemcpyAsync(exceed, dout, sizeof(float) * cells, cudaMemcpyDefault, s));
    if (n_levels)
        CK(g, cudaMemcpyAsync(pct, pct_dev, sizeof(float) * cells * n_levels, cudaMemcpyDefault, s));
    CK(g, cudaFreeAsync(buf, s));
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}
