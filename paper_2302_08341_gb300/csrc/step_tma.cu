// TMA-staged variant of the fused local-inertial step (same arithmetic and
// results, bit for bit, as step_kernel.cu).  Each warp owns one member's
// 128-column span of a strip of rows, as in the direct-load kernel, and
// streams its rows through shared memory (tma_march.cuh).
#include <cudaTypedefs.h>

#include "tma_march.cuh"

namespace flood {

namespace {

constexpr int kSpan = kTmaSpan;

// The land-cover form holds its class tables in registers: it gets more of
// them (four CTAs of four warps per SM instead of five) rather than spill.
// CK: the step may write checkpoints (the adjoint's logged forward); the
// ordinary step is compiled without that path.
template <int WM, bool TRACK_MAX, bool LC, int LIM, bool CK, bool HOOK = false>
__global__ void __launch_bounds__(32 * WM, (TRACK_MAX ? 16 : 20) / WM) step_tma_kernel(const __grid_constant__ TmaArgs t)
{
    extern __shared__ unsigned char smem_raw[];
    const StepArgs& a = t.a;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int m = blockIdx.x * WM + w;
    int span = blockIdx.y, strip = blockIdx.z;
    if (a.tiles) {  // only the tiles that hold a cell of the domain are launched
        const int2 tl = a.tiles[blockIdx.y];
        span = tl.x;
        strip = tl.y;
    }
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps; no block-wide barriers below
    if (*reinterpret_cast<volatile const int*>(a.err) & 2) return;  // an earlier wait gave up

    uint32_t bar0;
    unsigned char* my_stages;
    tma_march_smem(smem_raw, WM, w, bar0, my_stages, tma_stage_bytes(TRACK_MAX, LC));

    const size_t mstride = 3 * a.plane;
    // each warp is its own member here: the warp at the first span and strip owns its clock
    const MemberPlan pl = a.plan[m];
    if (!pl.active) return;
    float* __restrict__ dst = a.state + (size_t)((1 - pl.cur) * a.M + m) * mstride;
    float* ck = (CK && pl.ckpt >= 0) ? a.ckpt + ((size_t)pl.ckpt * a.M + m) * mstride : nullptr;

    FaceK k;
    k.gdt_dx = pl.gdt_dx;
    k.gdt = pl.gdt;
    k.dx_4dt = pl.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = pl.q_in;
    k.in_r0 = a.in_r0;
    k.in_r1 = a.in_r1;

    const int r0 = strip * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, a.ny);
    MarchOut mo;
    float* hm = TRACK_MAX ? a.hmax_field + (size_t)m * a.plane : nullptr;
    LandK lk;
    if (LC) lk = land_k(a, m, pl.dr, pl.dt, lane);
    if (!tma_march<TRACK_MAX, LC, LIM, HOOK>(&t.state_map, &t.static_map, (pl.cur * a.M + m) * 3, bar0,
                                  my_stages, dst, ck, hm, a.err, a.plane, a.ny, a.nx, a.ld, c0, r0,
                                  r1, lane, k, pl.dt_dx, a.scale[m], pl.dr, a.east_out, a.south_out,
                                  mo, &lk, a.wait_budget, &t.hm_map, m))
        return;

    if (mo.bad) atomicOr(a.err, 1);
    const unsigned hb = __reduce_max_sync(0xffffffffu, mo.bad ? 0u : __float_as_uint(mo.hmax) & 0x7fffffffu);
    double out_acc = (double)mo.out_s - (double)mo.out_c, clamp_acc = (double)mo.clamp;
    double drn_acc = LC ? (double)mo.drn_s - (double)mo.drn_c : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        out_acc += __shfl_xor_sync(0xffffffffu, out_acc, off);
        clamp_acc += __shfl_xor_sync(0xffffffffu, clamp_acc, off);
        if (LC) drn_acc += __shfl_xor_sync(0xffffffffu, drn_acc, off);
    }
    if (lane == 0) {
        atomicMax(&a.ms_out[m].hmax_bits, hb);
        const int slot = strip * ((a.nx + kSpan - 1) / kSpan) + span;
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            double* v = a.vacc + ((size_t)m * a.nslot + slot) * 2;
            v[0] += out_acc * pl.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
        if (LC && drn_acc != 0.0) a.dacc[(size_t)m * a.nslot + slot] += drn_acc * a.cell_area;
    }
}

// Replay of a logged step of a checkpointed segment for the adjoint: the
// same march as step_tma_kernel (so the recomputed states agree bit for bit
// with the forward's), reading the segment's slot replay_i and writing slot
// replay_i + 1, with the member's plan taken from the step log.  LC: with
// land cover (the class bytes ride in the stage, as in the step).
template <int WM, int LIM, bool LC = false>
__global__ void __launch_bounds__(32 * WM, 20 / WM) replay_tma_kernel(const __grid_constant__ TmaArgs t)
{
    extern __shared__ unsigned char smem_raw[];
    const StepArgs& a = t.a;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int m = blockIdx.x * WM + w;
    const int c0 = blockIdx.y * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps; no block-wide barriers below
    if (*reinterpret_cast<volatile const int*>(a.err) & 2) return;
    const int j = a.seg_first + a.replay_i;
    if (j >= a.seg_end[m]) return;

    uint32_t bar0;
    unsigned char* my_stages;
    tma_march_smem(smem_raw, WM, w, bar0, my_stages, tma_stage_bytes(false, LC));

    const size_t mstride = 3 * a.plane;
    const MemberPlan pl = a.log[(size_t)m * a.dt_log_cap + j];
    float* __restrict__ dst = a.seg + ((size_t)(a.replay_i + 1) * a.M + m) * mstride;
    FaceK k;
    k.gdt_dx = pl.gdt_dx;
    k.gdt = pl.gdt;
    k.dx_4dt = pl.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = pl.q_in;
    k.in_r0 = a.in_r0;
    k.in_r1 = a.in_r1;
    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, a.ny);
    MarchOut mo;
    LandK lk;
    if (LC) lk = land_k(a, m, pl.dr, pl.dt, lane);
    if (!tma_march<false, LC, LIM>(&t.state_map, &t.static_map, (a.replay_i * a.M + m) * 3, bar0,
                                   my_stages, dst, nullptr, nullptr, a.err, a.plane, a.ny, a.nx,
                                   a.ld, c0, r0, r1, lane, k, pl.dt_dx, a.scale[m], pl.dr,
                                   a.east_out, a.south_out, mo, &lk, kTmaWaitBudget, nullptr, 0))
        return;
    if (mo.bad) atomicOr(a.err, 1);
}

template <int WM, bool TRACK = false, bool LC = false>
size_t tma_smem_bytes()
{
    return tma_march_smem_bytes(WM, tma_stage_bytes(TRACK, LC));
}

}  // namespace

namespace {

// A tiled 3-D tensor map through the driver's encoder, obtained by the
// runtime's entry-point query (no link against libcuda).
int encode_map_3d_as(CUtensorMapDataType type, CUtensorMap* map, const void* base, uint64_t d0,
                     uint64_t d1, uint64_t d2, uint64_t stride1_bytes, uint64_t stride2_bytes,
                     uint32_t b0, uint32_t b1, uint32_t b2)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
    const cuuint32_t box[3] = {b0, b1, b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, type, 3, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace

int encode_map_3d(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                  uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t b0, uint32_t b1, uint32_t b2)
{
    return encode_map_3d_as(CU_TENSOR_MAP_DATA_TYPE_FLOAT32, map, base, d0, d1, d2, stride1_bytes,
                            stride2_bytes, b0, b1, b2);
}

int encode_map_3d_u8(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                     uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t b0, uint32_t b1,
                     uint32_t b2)
{
    return encode_map_3d_as(CU_TENSOR_MAP_DATA_TYPE_UINT8, map, base, d0, d1, d2, stride1_bytes,
                            stride2_bytes, b0, b1, b2);
}

int tma_box_cols() { return kTmaBox; }

namespace {

template <int WM, bool TRACK_MAX, bool LC, int LIM, bool CK, bool HOOK>
void launch_tma_wm(const TmaArgs& t, int spans, int strips, cudaStream_t s)
{
    static bool attr = false;
    const size_t shm = tma_smem_bytes<WM, TRACK_MAX, LC>();
    if (!attr) {
        cudaFuncSetAttribute(step_tma_kernel<WM, TRACK_MAX, LC, LIM, CK, HOOK>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        attr = true;
    }
    dim3 grid((t.a.M + WM - 1) / WM, spans, strips), block(32, WM);
    step_tma_kernel<WM, TRACK_MAX, LC, LIM, CK, HOOK><<<grid, block, shm, s>>>(t);
}

// Members per CTA: 4 or 1 for every variant; the plain step also has 2 and 8
// (the members-per-CTA sweep of the tuner and the benchmark).
template <bool TRACK_MAX, bool LC, int LIM, bool CK, bool HOOK = false>
void launch_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s)
{
    const StepArgs& a = t.a;
    const int spans = a.tiles ? a.n_tiles : (a.nx + kSpan - 1) / kSpan;
    const int strips = a.tiles ? 1 : (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    constexpr bool kPlain = !TRACK_MAX && !LC && !CK && !HOOK;
    if (kPlain && members_per_cta == 8)
        launch_tma_wm<kPlain ? 8 : 4, TRACK_MAX, LC, LIM, CK, HOOK>(t, spans, strips, s);
    else if (members_per_cta >= 4)
        launch_tma_wm<4, TRACK_MAX, LC, LIM, CK, HOOK>(t, spans, strips, s);
    else if (kPlain && members_per_cta == 2)
        launch_tma_wm<kPlain ? 2 : 1, TRACK_MAX, LC, LIM, CK, HOOK>(t, spans, strips, s);
    else
        launch_tma_wm<1, TRACK_MAX, LC, LIM, CK, HOOK>(t, spans, strips, s);
}

template <int LIM, bool LC>
void launch_replay_lim(const TmaArgs& t, int members_per_cta, cudaStream_t s)
{
    const StepArgs& a = t.a;
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        static bool attr = false;
        const size_t shm = tma_smem_bytes<4, false, LC>();
        if (!attr) {
            cudaFuncSetAttribute(replay_tma_kernel<4, LIM, LC>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            attr = true;
        }
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        replay_tma_kernel<4, LIM, LC><<<grid, block, shm, s>>>(t);
    } else {
        const size_t shm = tma_smem_bytes<1, false, LC>();
        dim3 grid(a.M, spans, strips), block(32, 1);
        replay_tma_kernel<1, LIM, LC><<<grid, block, shm, s>>>(t);
    }
}

}  // namespace

void launch_replay_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s)
{
    if (t.a.lc_on)
        t.a.limiter ? launch_replay_lim<1, true>(t, members_per_cta, s)
                    : launch_replay_lim<0, true>(t, members_per_cta, s);
    else
        t.a.limiter ? launch_replay_lim<1, false>(t, members_per_cta, s)
                    : launch_replay_lim<0, false>(t, members_per_cta, s);
}

int launch_step_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s)
{
    const bool track = t.a.hmax_field != nullptr;
    const bool lim = t.a.limiter != 0;
    if (t.a.wait_budget != kTmaWaitBudgetDefault) {  // the failure-detection hook: plain step only
        if (track || t.a.lc_on || t.a.ckpt) return -1;
        lim ? launch_tma<false, false, 1, false, true>(t, members_per_cta, s)
            : launch_tma<false, false, 0, false, true>(t, members_per_cta, s);
        return 0;
    }
    if (t.a.ckpt) {  // the adjoint's logged forward
        if (t.a.lc_on) {
            if (track)
                lim ? launch_tma<true, true, 1, true>(t, members_per_cta, s)
                    : launch_tma<true, true, 0, true>(t, members_per_cta, s);
            else
                lim ? launch_tma<false, true, 1, true>(t, members_per_cta, s)
                    : launch_tma<false, true, 0, true>(t, members_per_cta, s);
        } else if (track)
            lim ? launch_tma<true, false, 1, true>(t, members_per_cta, s)
                : launch_tma<true, false, 0, true>(t, members_per_cta, s);
        else
            lim ? launch_tma<false, false, 1, true>(t, members_per_cta, s)
                : launch_tma<false, false, 0, true>(t, members_per_cta, s);
    } else if (t.a.lc_on) {
        if (track)
            lim ? launch_tma<true, true, 1, false>(t, members_per_cta, s)
                : launch_tma<true, true, 0, false>(t, members_per_cta, s);
        else
            lim ? launch_tma<false, true, 1, false>(t, members_per_cta, s)
                : launch_tma<false, true, 0, false>(t, members_per_cta, s);
    } else {
        if (track)
            lim ? launch_tma<true, false, 1, false>(t, members_per_cta, s)
                : launch_tma<true, false, 0, false>(t, members_per_cta, s);
        else
            lim ? launch_tma<false, false, 1, false>(t, members_per_cta, s)
                : launch_tma<false, false, 0, false>(t, members_per_cta, s);
    }
    return 0;
}

}  // namespace flood
