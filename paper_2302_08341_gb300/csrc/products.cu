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
#include <cstring>
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
    uint32_t th_ord;      // ord of the threshold (of -0 for a zero threshold): x >= it iff ord(x) >= th_ord
    int n_levels;                  // levels of this pass (<= kLevelsPerPass)
    long long A[kLevelsPerPass];   // level thresholds in units of 2^-60
    int rank[kLevelsPerPass];      // equal weights: 1-based rank reaching the level (M + 1: none)
    long long u_eq;                // equal weights: the common weight
    float* exceed;        // [ny][nx] (or null)
    float* pct;           // [n_levels][ny][nx] of this pass (or null)
    int* err;             // the grid's error word (bit 1: a bounded wait gave up)
};

__device__ __forceinline__ float exceed_value(long long units)
{
    return (float)(__ll2double_rn(units) * 0x1p-60);
}

// Batcher's odd-even merge sort on N (a power of two) slots, every
// comparator ascending (min to the lower slot).  Slots MT..N-1 would hold
// the largest value and never move, so every comparator reaching them is
// left out: the network sorts MT slots.  The merge levels (P, K) are
// template parameters, so every slot index is a compile-time constant and
// the slots stay in registers.  The slots are FP32 values (equal weights)
// or 32-bit keys (below).
__device__ __forceinline__ void order2(float& x, float& y)
{
    const float lo = fminf(x, y);
    y = fmaxf(x, y);
    x = lo;
}
__device__ __forceinline__ void order2(uint32_t& x, uint32_t& y)
{
    const uint32_t lo = min(x, y);
    y = max(x, y);
    x = lo;
}

template <typename T, int N, int MT, int P, int K>
__device__ __forceinline__ void merge_level(T (&v)[MT])
{
#pragma unroll
    for (int j = K % P; j + K < N; j += 2 * K) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (i + j + K < MT && (i + j) / (2 * P) == (i + j + K) / (2 * P))
                order2(v[i + j], v[i + j + K]);
        }
    }
    if constexpr (K > 1) merge_level<T, N, MT, P, K / 2>(v);
}

template <typename T, int N, int MT, int P = 1>
__device__ __forceinline__ void odd_even_merge_sort(T (&v)[MT])
{
    if constexpr (P < N) {
        merge_level<T, N, MT, P, P>(v);
        odd_even_merge_sort<T, N, MT, 2 * P>(v);
    }
}

// An order-preserving map of FP32 bit patterns onto unsigned integers
// (negative values reversed below the positive ones): for non-NaN x, y
// other than the pair -0, +0, x < y iff ord(x) < ord(y); ord(-0) is one
// below ord(+0).
__device__ __forceinline__ uint32_t ord_of(float x)
{
    const uint32_t b = __float_as_uint(x);
    return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
}
__device__ __forceinline__ float from_ord(uint32_t o)
{
    return __uint_as_float(o ^ ((uint32_t)((int32_t)~o >> 31) | 0x80000000u));
}

// Arguments of the staged kernel: the running maxima as a 3-D tensor map
// (nx, ny, M) whose box is 32 cells x 1 row x M members (one warp's group),
// and the cell groups (32 consecutive cells of one row) to cover.
struct ProdTma {
    CUtensorMap map;
    ProdArgs a;
    int n_groups, groups_per_row;
};

constexpr int kProdWarps = 4;  // warps per CTA of the staged kernel

template <int MT>
__host__ __device__ constexpr int prod_stage_bytes() { return (MT * 32 * 4 + 127) / 128 * 128; }

// One thread per cell, warps persistent over groups of 32 cells.  A group's
// maxima (every member of 32 cells) arrive by one tensor copy into the
// warp's stage; the lanes read them into registers, sort them there, and
// write the sorted slots back into their own columns of the stage, from
// which the levels are read; then the copy of the warp's next group starts
// (the other warps of the SM cover its latency).
//
// Equal weights: the cell's MT slots (members, then +inf padding) are
// sorted as FP32 values and the a-percentile is the value of the rank that
// first reaches a (ranks from the host).  Tied values may come out in any
// order: the first position to reach a level then still holds the tied
// value.
//
// Unequal weights: each member becomes one 32-bit key, its value's place
// above the cell's smallest value in the high 25 bits and its index in the
// low 7, so sorting the keys as integers orders the members and carries
// their indices at the cost of a value sort.  The place is ord(x) - ord(min),
// exact while the cell's values span fewer than 2^25 - 1 representable
// FP32 numbers (about four binades); beyond that it is shifted right by the
// fewest bits that fit, so values closer than 2^shift representable numbers
// may share a place and come out in index order.  One pass over the sorted
// keys sums the weights (exact integers) and keeps, per level, the key at
// the first position whose cumulative weight reaches it, and the weight of
// the members at or above the threshold.  A lane with shifted places then
// checks its sorted keys: a level whose key is alone in its place takes that
// member's value from its maxima in global memory; where members share it,
// the answer lies among them (every place below holds smaller values, every
// place above larger ones), and candidates are tried in increasing order
// against the exact weighted distribution function.  The members in the
// threshold's place, counted as reaching it, are checked against it.
//
// Every wait is bounded: one that gives up records FLOOD_ERR_TIMEOUT in the
// error word, waits for the warp's copy in flight and returns.
template <int MT, bool EQUAL>
__global__ void __launch_bounds__(32 * kProdWarps, MT <= 96 ? 4 : 2)
    tma_products_kernel(const __grid_constant__ ProdTma t)
{
    extern __shared__ unsigned char smem_raw[];
    const ProdArgs& a = t.a;
    constexpr int kStage = prod_stage_bytes<MT>();
    constexpr long long kBudget = flood::kTmaWaitBudgetDefault;
    constexpr uint32_t kPad = 0xFFFFFFFFu;   // key of a padding slot: index 127, no weight
    __shared__ long long us[EQUAL ? 1 : 128];
    if (!EQUAL) {
        for (int j = threadIdx.x; j < 128; j += blockDim.x) us[j] = j < a.M ? a.u[j] : 0;
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    const uint32_t bar = flood::smem_u32(base) + 8u * w;
    float* const stage = reinterpret_cast<float*>(base + 128 + kStage * w);
    const uint32_t stage_s = flood::smem_u32(stage);
    const uint32_t tx = 32u * 4u * (uint32_t)a.M;
    const int gw = blockIdx.x * kProdWarps + w, nwarps = gridDim.x * kProdWarps;
    if (lane == 0) {
        flood::mbar_init(bar, 1);
        flood::fence_mbar_init();
    }
    __syncwarp();
    auto issue = [&](int g) {
        const int r = g / t.groups_per_row, c0 = (g % t.groups_per_row) * 32;
        flood::mbar_arrive_expect_tx(bar, tx);
        flood::tma_load_3d(stage_s, &t.map, c0, r, 0, bar);
    };
    // the next group's copy, once every lane has read the stage
    auto release = [&](int g) {
        __syncwarp();
        const int gn = g + nwarps;
        if (gn < t.n_groups && lane == 0) {
            flood::fence_proxy_async_smem();
            issue(gn);
        }
    };
    if (gw < t.n_groups && lane == 0) issue(gw);
    uint32_t phase = 0;
    constexpr int N = MT <= 32 ? 32 : MT <= 64 ? 64 : 128;   // the network's power of two
    constexpr int kStep = MT >= 128 ? 128 : MT >= 64 ? 64 : 32;  // largest power of two <= MT
    for (int g = gw; g < t.n_groups; g += nwarps) {
        if (!flood::mbar_wait_bounded(bar, phase, kBudget)) {
            if (lane == 0) atomicOr(a.err, 2);
            flood::mbar_wait_bounded(bar, phase, kBudget);  // the copy in flight lands first
            return;
        }
        phase ^= 1u;
        const int r = g / t.groups_per_row, c = (g % t.groups_per_row) * 32 + lane;
        const size_t out = (size_t)r * a.nx + c;
        if constexpr (EQUAL) {
            float v[MT];
#pragma unroll
            for (int j = 0; j < MT; ++j)
                v[j] = j < a.M ? stage[j * 32 + lane] : __int_as_float(0x7f800000);
            odd_even_merge_sort<float, N, MT>(v);
            // the sorted slots go back into this lane's column of the stage
            // (the lane alone reads and writes it): a level then reads one
            // word, and the members below the threshold are a binary search
            // on the column (the +inf padding is never below it), where
            // reading v[k] for a run-time k would take a select per slot
            float* const col = stage + lane;
#pragma unroll
            for (int k = 0; k < MT; ++k) col[k * 32] = v[k];
            int below = 0;  // the sorted slots below the threshold, a prefix of the column
#pragma unroll
            for (int st = kStep; st > 0; st >>= 1)
                if (below + st <= MT && col[(below + st - 1) * 32] < a.threshold) below += st;
            const int cnt = a.M - below;
            float pv[kLevelsPerPass];
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q)  // rank past M: none reaches the level, the top
                pv[q] = col[min(a.rank[q] - 1, a.M - 1) * 32];
            release(g);
            if (c >= a.nx) continue;
            if (a.exceed) a.exceed[out] = exceed_value((long long)cnt * a.u_eq);
            if (!a.pct) continue;
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q) {
                if (q >= a.n_levels) break;
                a.pct[(size_t)q * a.ny * a.nx + out] = pv[q];
            }
        } else {
            uint32_t key[MT];
            uint32_t omin = kPad, omax = 0u;
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                if (j < a.M) {
                    const uint32_t o = ord_of(stage[j * 32 + lane]);
                    key[j] = o;
                    omin = min(omin, o);
                    omax = max(omax, o);
                } else {
                    key[j] = kPad;
                }
            }
            const uint32_t d = omax - omin;
            int sh = max(0, 7 - __clz(d));              // bits of d above 25
            if ((d >> sh) == 0x1FFFFFFu) ++sh;          // keeps real keys below kPad
            const bool exact = sh == 0;
#pragma unroll
            for (int j = 0; j < MT; ++j)
                if (j < a.M) key[j] = (((key[j] - omin) >> sh) << 7) | (uint32_t)j;
            odd_even_merge_sort<uint32_t, N, MT>(key);
            // the sorted keys go into this lane's column of the stage (its
            // values are in registers now), and the pass over them is a short
            // loop: unrolled over the registers it doubled the code and the
            // warps waited on instruction fetch
            uint32_t* const kcol = reinterpret_cast<uint32_t*>(stage) + lane;
#pragma unroll
            for (int k = 0; k < MT; ++k) kcol[k * 32] = key[k];
            // the threshold as a key: the first key of its place (shifted
            // lanes settle the members of that place below)
            const uint32_t kth =
                a.th_ord <= omin ? 0u : a.th_ord > omax ? kPad : ((a.th_ord - omin) >> sh) << 7;
            long long P = 0, ex = 0;
            uint32_t kc[kLevelsPerPass];
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q) kc[q] = kPad;
#pragma unroll 4
            for (int k = 0; k < MT; ++k) {
                const uint32_t kk = kcol[k * 32];
                const long long uk = us[kk & 0x7Fu];
#pragma unroll
                for (int q = 0; q < kLevelsPerPass; ++q) kc[q] = P < a.A[q] ? kk : kc[q];
                P += uk;
                ex += kk >= kth ? uk : 0;
            }
            // per level the ord of the answer (none reached: the largest value)
            uint32_t oq[kLevelsPerPass];
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q) oq[q] = P < a.A[q] ? omax : (kc[q] >> 7) + omin;
            if (!exact) {
                // a lane with shifted places: its keys order the members up
                // to values that share a place.  The exceedance counted every
                // member in the threshold's place as reaching it, and a level
                // whose key shares its place with other members needs their
                // values: both are settled from the maxima in global memory
                // (the stage holds the keys now; the group's lines are still
                // in L2)
                const float* fc = a.field + (size_t)r * a.ld + c;
                auto below_key = [&](uint32_t kq) -> int {  // sorted keys below kq
                    int n = 0;
#pragma unroll
                    for (int st = kStep; st > 0; st >>= 1)
                        if (n + st <= MT && kcol[(n + st - 1) * 32] < kq) n += st;
                    return n;
                };
                if (a.th_ord > omin && a.th_ord <= omax) {
                    const uint32_t pth = (a.th_ord - omin) >> sh;
                    const int end = below_key((pth + 1) << 7);
                    for (int p = below_key(pth << 7); p < end; ++p) {
                        const uint32_t id = kcol[p * 32] & 0x7Fu;  // a real member: < M
                        if (id < (uint32_t)a.M && ord_of(fc[(size_t)id * a.plane]) < a.th_ord) ex -= us[id];
                    }
                }
#pragma unroll
                for (int q = 0; q < kLevelsPerPass; ++q) {
                    if (q >= a.n_levels || P < a.A[q]) continue;
                    const uint32_t pl = kc[q] >> 7;
                    const int plo = below_key(pl << 7), phi = below_key((pl + 1) << 7);
                    if (phi - plo == 1) {  // the key's member is alone in its place
                        oq[q] = ord_of(fc[(size_t)min(kc[q] & 0x7Fu, (uint32_t)a.M - 1u) * a.plane]);
                        continue;
                    }
                    // members that share the place: their range, then
                    // candidates in increasing order against the exact
                    // weighted distribution function (lower places hold
                    // smaller values, higher places larger ones)
                    uint32_t lo = kPad, hi = 0u;
                    for (int p = plo; p < phi; ++p) {
                        const uint32_t id = min(kcol[p * 32] & 0x7Fu, (uint32_t)a.M - 1u);
                        const uint32_t o = ord_of(fc[(size_t)id * a.plane]);
                        lo = min(lo, o);
                        hi = max(hi, o);
                    }
                    uint32_t v = lo;
                    for (int it = 0; it < a.M && v != hi; ++it) {
                        long long W = 0;
                        uint32_t nxt = hi;
                        for (int j = 0; j < a.M; ++j) {
                            const uint32_t o = ord_of(fc[(size_t)j * a.plane]);
                            if (o <= v) W += us[j];
                            else nxt = min(nxt, o);
                        }
                        if (W >= a.A[q]) break;
                        v = nxt;
                    }
                    oq[q] = v;
                }
            }
            // the shifted lanes have read the keys: the next copy may overwrite them
            release(g);
            if (c >= a.nx) continue;
            if (a.exceed) a.exceed[out] = exceed_value(ex);
            if (!a.pct) continue;
#pragma unroll
            for (int q = 0; q < kLevelsPerPass; ++q) {
                if (q >= a.n_levels) break;
                a.pct[(size_t)q * a.ny * a.nx + out] = from_ord(oq[q]);
            }
        }
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
void launch_tma_products(ProdTma& t, int n_sm, cudaStream_t s)
{
    constexpr size_t shm = 128 + (size_t)prod_stage_bytes<MT>() * kProdWarps + 128;
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(tma_products_kernel<MT, EQUAL>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tma_products_kernel<MT, EQUAL>,
                                                      32 * kProdWarps, shm);
        per_sm = std::max(per_sm, 1);
    }
    const int need = (t.n_groups + kProdWarps - 1) / kProdWarps;
    const int blocks = std::max(1, std::min(need, n_sm * per_sm));
    tma_products_kernel<MT, EQUAL><<<blocks, 32 * kProdWarps, shm, s>>>(t);
}

// The staged kernel up to 128 members (its copy box holds every member of
// 32 cells), the shared-memory kernel beyond or without a tensor map.
void launch_products(ProdTma& t, bool have_map, bool equal, int n_sm, cudaStream_t s)
{
    const int M = t.a.M;
    if (!have_map || M > 128) {
        dim3 grid((t.a.nx + kCells - 1) / kCells, t.a.ny);
        staged_products_kernel<<<grid, kCells, products_smem(M), s>>>(t.a);
    } else if (equal) {
        if (M <= 32) launch_tma_products<32, true>(t, n_sm, s);
        else if (M <= 64) launch_tma_products<64, true>(t, n_sm, s);
        else if (M <= 96) launch_tma_products<96, true>(t, n_sm, s);
        else launch_tma_products<128, true>(t, n_sm, s);
    } else {
        if (M <= 32) launch_tma_products<32, false>(t, n_sm, s);
        else if (M <= 64) launch_tma_products<64, false>(t, n_sm, s);
        else if (M <= 96) launch_tma_products<96, false>(t, n_sm, s);
        else launch_tma_products<128, false>(t, n_sm, s);
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
    // outputs in device memory are written in place; others go through a
    // device buffer and a copy
    auto on_device = [](const void* p) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    };
    const bool ex_dev = exceed && on_device(exceed);
    const bool pct_dev_ok = n_levels > 0 && on_device(pct);
    const size_t need_f = (exceed && !ex_dev ? cells : 0) + (pct_dev_ok ? 0 : (size_t)n_levels * cells);
    char* buf = nullptr;
    if (need_f) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), sizeof(float) * need_f, s);
        if (e != cudaSuccess)
            return flood::fail(g, e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA,
                               std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    float* dtmp = reinterpret_cast<float*>(buf);
    float* dex = ex_dev ? exceed : (exceed ? dtmp : nullptr);
    float* dpct = pct_dev_ok ? pct : (n_levels ? dtmp + (exceed && !ex_dev ? cells : 0) : nullptr);
    if (!g->prod_u) {
        const int rc = flood::dalloc(g, &g->prod_u, kMaxMembers);
        if (rc) return rc;
    }
    long long* du = g->prod_u;
    CK(g, cudaMemcpyAsync(du, u.data(), sizeof(long long) * M, cudaMemcpyHostToDevice, s));
    static bool attr = false;
    if (!attr) {
        CK(g, cudaFuncSetAttribute(staged_products_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)products_smem(kMaxMembers)));
        attr = true;
    }
    // the maxima as (nx, ny, M) with a box of 32 cells x 1 row x M members
    ProdTma tm{};
    const bool have_map =
        M <= 128 && flood::encode_map_3d(&tm.map, g->hmax_field, g->nx, g->ny, (uint64_t)M,
                                         sizeof(float) * g->ld, sizeof(float) * g->plane, 32, 1,
                                         (uint32_t)M) == 0;
    tm.groups_per_row = (g->nx + 31) / 32;
    tm.n_groups = tm.groups_per_row * g->ny;
    ProdArgs& a = tm.a;
    a.err = g->err;
    a.field = g->hmax_field;
    a.u = du;
    a.M = M;
    a.ny = g->ny; a.nx = g->nx; a.ld = g->ld;
    a.plane = g->plane;
    a.threshold = (float)threshold;
    {
        // the order-preserving map of the kernels' keys; a zero threshold
        // takes ord(-0), so that -0 and +0 both reach it
        uint32_t b = 0;
        std::memcpy(&b, &a.threshold, 4);
        a.th_ord = a.threshold == 0.0f ? 0x7FFFFFFFu : b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
    }
    a.u_eq = u[0];
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
        a.exceed = q0 == 0 ? dex : nullptr;
        a.pct = a.n_levels > 0 ? dpct + (size_t)q0 * cells : nullptr;
        launch_products(tm, have_map, equal, g->n_sm, s);
        g->launches++;
        CK(g, cudaGetLastError());
    }
    if (exceed && !ex_dev) CK(g, cudaMemcpyAsync(exceed, dex, sizeof(float) * cells, cudaMemcpyDefault, s));
    if (n_levels && !pct_dev_ok)
        CK(g, cudaMemcpyAsync(pct, dpct, sizeof(float) * cells * n_levels, cudaMemcpyDefault, s));
    if (buf) CK(g, cudaFreeAsync(buf, s));
    CK(g, cudaStreamSynchronize(s));
    int err = 0;
    CK(g, cudaMemcpy(&err, g->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 2) return flood::fail(g, FLOOD_ERR_TIMEOUT, "a bounded wait for staged maxima gave up");
    return FLOOD_OK;
}
