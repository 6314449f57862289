// The TMA-staged march of one warp over a 128-column span of rows
// [r0, r1) of one grid (an ensemble member or a batched scenario), shared by
// the ensemble (step_tma.cu) and batched (batch_kernel.cu) step kernels.
//
// The warp's rows arrive through a ring of kTmaNS shared-memory stages filled
// by the tensor memory accelerator: one 3-D tiled copy brings a row of h, qx
// and qy (136 columns: the span plus 4 halo columns each side, zero-filled
// past the grid's edges), another the same row of z and n.  Lane 0 keeps
// kTmaNS - 1 rows in flight ahead of the row being computed, so the memory
// latency is covered by the warp's own pipeline; the halo comes with the
// tile, so no scalar edge loads remain.  Every mbarrier wait is bounded: on
// timeout the march records FLOOD_ERR_TIMEOUT in the error word, waits
// (bounded) for its own copies in flight, and returns false.
#pragma once

#include "march.cuh"
#include "tma.cuh"

namespace flood {

constexpr int kTmaSpan = 128;
constexpr int kTmaNS = 4;                          // stages per warp
constexpr int kTmaBox = kTmaSpan + 8;              // columns per tile row
constexpr int kTmaStaticOff = 1664;                // bytes: z, n after h, qx, qy (128-aligned)
constexpr int kTmaStageBytes = 2816;               // 128-aligned stage size
constexpr uint32_t kTmaTx = kTmaBox * 3 * 4 + kTmaBox * 2 * 4;  // bytes landing per stage
constexpr long long kTmaWaitBudget = kTmaWaitBudgetDefault;  // clock cycles before giving up
static_assert((kTmaNS & (kTmaNS - 1)) == 0, "ring index arithmetic needs a power of two");

// Dynamic shared memory of a CTA of `warps` warps: barriers, then each warp's
// stages.
__host__ __device__ constexpr size_t tma_march_smem_bytes(int warps, int stage_bytes = kTmaStageBytes)
{
    return 128 + 128 * ((8 * kTmaNS * warps + 127) / 128) + (size_t)kTmaNS * stage_bytes * warps;
}
constexpr int kTmaHmOff = kTmaStageBytes;              // running maxima: 128 floats after z, n
// With land cover the static planes are the bed and each cell's class code
// (a uint32 where the roughness would be): the stage keeps its size.
__host__ __device__ constexpr int tma_stage_bytes(bool track, bool lc)
{
    return kTmaStageBytes + (track ? 512 : 0) + (lc ? 0 : 0);
}

// This warp's barriers and stages inside the CTA's dynamic shared memory.
__device__ __forceinline__ void tma_march_smem(unsigned char* smem_raw, int warps, int w,
                                               uint32_t& bar0, unsigned char*& my_stages,
                                               int stage_bytes = kTmaStageBytes)
{
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    bar0 = smem_u32(base) + 8u * kTmaNS * w;
    my_stages = base + 128 * ((8 * kTmaNS * warps + 127) / 128) + kTmaNS * stage_bytes * w;
}

__device__ __forceinline__ void tma_lds4(float (&v)[4], const float* p)
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void tma_store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// state_map: (ld, ny, planes) with the source h, qx, qy at planes
// [plane0, plane0 + 3); static_map: (ld, ny, 2) with z then n.  Writes the
// new state to dst (and ck when non-null); TRACK_MAX: also raises the
// running maximum depth at hm, whose old values arrive with each row through
// hm_map (member plane hm_plane, 128 columns from c0; a 3.3 KB stage, so four
// CTAs of four warps per SM); LC: land cover (roughness by class from lk,
// the class's share of the rain and its drainage; static_map then holds the
// bed and each cell's class code, so the codes arrive with the row where
// the roughness would, halo included).  Each is a separate
// instantiation, so the plain step carries no trace of them.  Returns false
// if a wait gave up.  WAIT_HOOK: each row wait may take wait_budget clock
// cycles instead of kTmaWaitBudget (a failure-detection hook; the copies
// still in flight are always drained with the full kTmaWaitBudget).
template <bool TRACK_MAX, bool LC = false, int LIM = -1, bool WAIT_HOOK = false>
__device__ __forceinline__ bool tma_march(const CUtensorMap* state_map, const CUtensorMap* static_map,
                                          int plane0, uint32_t bar0, unsigned char* my_stages,
                                          float* __restrict__ dst, float* ck, float* hm, int* err,
                                          size_t plane,
                                          int ny, int nx, int ld, int c0, int r0, int r1, int lane,
                                          const FaceK& k, float dt_dx, float s, float dr,
                                          int east_out, int south_out, MarchOut& out,
                                          const LandK* lk = nullptr,
                                          long long wait_budget = kTmaWaitBudget,
                                          const CUtensorMap* hm_map = nullptr, int hm_plane = 0)
{
    constexpr int kNS = kTmaNS;
    constexpr int kBox = kTmaBox;
    constexpr int kStaticOff = kTmaStaticOff;
    constexpr int kStageBytes = tma_stage_bytes(TRACK_MAX, LC);
    constexpr uint32_t kTx = kTmaTx + (TRACK_MAX ? 512u : 0u);
    constexpr int kZ = kStaticOff / 4;
    constexpr int kN = kZ + kBox;
    constexpr long long kWaitBudget = kTmaWaitBudget;
    const uint32_t stage0 = smem_u32(my_stages);
    const float s_half = 0.5f * s;

    const int c = c0 + 4 * lane;
    const bool act = c < nx;
    const bool interior = (c + 4 < nx);
    const bool edge_warp = c0 + kTmaSpan >= nx;  // the span holds the grid's last column
    const int ra = r0 > 0 ? r0 - 1 : r0;   // first row loaded
    const int rb = min(r1 + 1, ny);        // one past the last row loaded

    if (lane == 0) {
        for (int i = 0; i < kNS; ++i) mbar_init(bar0 + 8u * i, 1);
        fence_mbar_init();
    }
    __syncwarp();
    int issued = ra;  // rows [ra, issued) have been requested
    auto issue = [&](int row) {
        const unsigned sidx = (unsigned)(row - ra) & (kNS - 1);
        const uint32_t bar = bar0 + 8u * sidx;
        const uint32_t dsts = stage0 + kStageBytes * sidx;
        mbar_arrive_expect_tx(bar, kTx);
        tma_load_3d(dsts, state_map, c0 - 4, row, plane0, bar);
        tma_load_3d(dsts + kStaticOff, static_map, c0 - 4, row, 0, bar);
        if (TRACK_MAX) tma_load_3d(dsts + kTmaHmOff, hm_map, c0, row, hm_plane, bar);
    };
    // land classes of a staged row (LC: the class-code plane): the lane's
    // four cells as one byte each of a word
    auto cls_of = [&](const float* P) -> uint32_t {
        const uint4 q = *reinterpret_cast<const uint4*>(P + kN + 4 + 4 * lane);
        return __byte_perm(__byte_perm(q.x, q.y, 0x0040u), __byte_perm(q.z, q.w, 0x0040u), 0x5410u);
    };
    for (; issued < rb && issued < ra + kNS; ++issued)
        if (lane == 0) issue(issued);
    auto wait_row_for = [&](int row, long long budget) -> bool {
        const int kk = row - ra;
        return mbar_wait_bounded(bar0 + 8u * ((unsigned)kk & (kNS - 1)), ((unsigned)kk / kNS) & 1,
                                 budget);
    };
    auto wait_row = [&](int row) -> bool {
        return wait_row_for(row, WAIT_HOOK ? wait_budget : kWaitBudget);
    };
    auto row_ptr = [&](int row) -> const float* {
        return reinterpret_cast<const float*>(my_stages +
                                              kStageBytes * ((unsigned)(row - ra) & (kNS - 1)));
    };
    // recycle the stage of `row` for the next row in line
    auto release = [&](int row) {
        __syncwarp();
        if (issued < rb) {
            if (lane == 0) {
                fence_proxy_async_smem();
                issue(issued);
            }
            ++issued;
        }
        (void)row;
    };
    int waited = ra;  // rows [ra, waited) have landed
    bool ok = true;
    auto drain_and_fail = [&]() {
        if (lane == 0) atomicOr(err, 2);
        // every copy still in flight lands before the warp leaves (bounded each)
        for (int row = waited; row < issued; ++row) wait_row_for(row, kWaitBudget);
    };

    const int x0 = 4 + 4 * lane;  // this lane's first cell in a tile row
    float hC[4] = {0, 0, 0, 0}, zC[4] = {0, 0, 0, 0}, nC[4] = {0, 0, 0, 0};
    float qyN[4] = {0, 0, 0, 0};
    if (r0 > 0) {
        ok = wait_row(r0 - 1);
        if (ok) waited = r0;
    }
    if (ok) {
        ok = wait_row(r0);
        if (ok) waited = r0 + 1;
    }
    if (!ok) {
        drain_and_fail();
        return false;
    }
    // land classes (LC): they come with each staged row (zeros past the
    // grid's edges, where no link uses them)
    uint32_t clsC = 0;
    {
        const float* P = row_ptr(r0);
        if (LC) clsC = cls_of(P);
        tma_lds4(hC, P + x0);
        tma_lds4(zC, P + kZ + x0);
        if (LC)
            land_n4(nC, clsC, *lk);
        else
            tma_lds4(nC, P + kN + x0);
        if (r0 > 0) {
            const float* U = row_ptr(r0 - 1);
            float hU[4], zU[4], nU[4], qU[4];
            tma_lds4(hU, U + x0);
            tma_lds4(zU, U + kZ + x0);
            if (LC)  // whole warp: the lookups are shuffles
                land_n4(nU, cls_of(U), *lk);
            else
                tma_lds4(nU, U + kN + x0);
            tma_lds4(qU, U + 2 * kBox + x0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                qyN[j] = (c + j < nx)
                             ? link_q<LIM>(hU[j], zU[j], hC[j], zC[j], qU[j],
                                      __fmul_rn(s_half, __fadd_rn(nU[j], nC[j])), k)
                             : 0.0f;
            release(r0 - 1);
        }
    }

    float hmax = 0.0f;
    float out_s = 0.0f, out_c = 0.0f, clamp = 0.0f, drn_s = 0.0f, drn_c = 0.0f;

#pragma unroll 2
    for (int r = r0; r < r1; ++r) {
        const size_t o = (size_t)r * ld + c;
        const bool has_s = (r + 1 < ny);
        if (has_s) {
            if (!wait_row(r + 1)) {
                drain_and_fail();
                return false;
            }
            waited = r + 2;
        }
        const float* P = row_ptr(r);
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0};
        float qxo[4], qyo[4];
        float4 hmo = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (TRACK_MAX) hmo = *reinterpret_cast<const float4*>(P + kTmaHmOff / 4 + 4 * lane);
        tma_lds4(qxo, P + kBox + x0);
        tma_lds4(qyo, P + 2 * kBox + x0);
        uint32_t clsS = 0;
        if (LC) {
            // the whole warp, outside any branch (the lookups are shuffles);
            // past the grid's last row the stage holds an earlier row, whose
            // classes go unused
            clsS = cls_of(row_ptr(r + 1));
            land_n4(nS, clsS, *lk);
        }
        if (has_s) {
            const float* Q = row_ptr(r + 1);
            tma_lds4(hS, Q + x0);
            tma_lds4(zS, Q + kZ + x0);
            if (!LC) tma_lds4(nS, Q + kN + x0);
        }
        // east neighbour of the lane's last cell, straight from the tile
        const float hE = P[x0 + 4], zE = P[kZ + x0 + 4];
        float nE;
        float nWl = 0.0f, drv[4], ddv[4];
        if (LC) {
            // the east neighbour's and the west halo cell's classes come
            // with the tile (the codes sit where the roughness would)
            nE = land_get(lk->n, __float_as_uint(P[kN + x0 + 4]));
            nWl = land_get(lk->n, __float_as_uint(P[kN + 3]));
            land_src4(drv, ddv, clsC, *lk);
        } else {
            nE = P[kN + x0 + 4];
        }
        float qxE[4], qyS[4];
        if (interior)
            row_links<true, LIM>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                            east_out, south_out, qxE, qyS);
        else
            row_links<false, LIM>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                             east_out, south_out, qxE, qyS);
        float qW0 = __shfl_up_sync(0xffffffffu, qxE[3], 1);
        if (lane == 0) {
            qW0 = (r >= k.in_r0 && r < k.in_r1) ? k.q_in : 0.0f;  // west edge: wall or inflow
            if (c0 > 0) {  // the neighbouring span's last link, from the tile's halo
                const float nW = LC ? nWl : P[kN + 3];
                qW0 = link_q<LIM>(P[3], P[kZ + 3], hC[0], zC[0], P[kBox + 3],
                             __fmul_rn(s_half, __fadd_rn(nW, nC[0])), k);
            }
        }
        float hN[4];
        if (interior)
            row_depths<true, LC>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hN,
                                 drv, ddv, &drn_s, &drn_c);
        else
            row_depths<false, LC>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hN,
                                  drv, ddv, &drn_s, &drn_c);
        if ((edge_warp && east_out) || (!has_s && south_out)) {  // the same for the whole warp
            // links leaving the domain this row: the east edge link (one lane)
            // and, on the last row, the south edge links
            float ev = 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + j == nx - 1 && east_out) ev = qxE[j];
            if (!has_s && south_out)
                ev = __fadd_rn(ev, __fadd_rn(__fadd_rn(qyS[0], qyS[1]), __fadd_rn(qyS[2], qyS[3])));
            kahan_add(out_s, out_c, ev);
        }
        if (act) {
            tma_store4(dst + o, hN);
            tma_store4(dst + plane + o, qxE);
            tma_store4(dst + 2 * plane + o, qyS);
            if (ck) {
                tma_store4(ck + o, hN);
                tma_store4(ck + plane + o, qxE);
                tma_store4(ck + 2 * plane + o, qyS);
            }
            if (TRACK_MAX)
                *reinterpret_cast<float4*>(hm + o) =
                    make_float4(fmaxf(hmo.x, hN[0]), fmaxf(hmo.y, hN[1]), fmaxf(hmo.z, hN[2]),
                                fmaxf(hmo.w, hN[3]));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            qyN[j] = qyS[j];
            hC[j] = hS[j];
            zC[j] = zS[j];
            nC[j] = nS[j];
        }
        clsC = clsS;
        release(r);
    }

    out.hmax = hmax;
    out.bad = !(hmax <= 3.0e38f);  // a NaN or an overflow anywhere
    out.out_s = out_s;
    out.out_c = out_c;
    out.clamp = clamp;
    out.drn_s = drn_s;
    out.drn_c = drn_c;
    return true;
}

}  // namespace flood
