// Per-warp march of the fused step over one 128-column span of rows
// [r0, r1) of one member: reads the state at src (h, qx, qy planes) and the
// shared z, n; writes the new state to dst (and ck when non-null), raises the
// running maximum depth at hm (when non-null) to the new depth; returns
// the warp-local maximum depth, the non-finite flag and the outflow / clamp
// partial sums.  Shared by the ensemble, replay and batched step kernels.
#pragma once

#include "flood_internal.cuh"

namespace flood {

struct MarchOut {
    float hmax;
    bool bad;
    float out_s, out_c;   // outflow sum of q over the warp's edge links (Kahan pair)
    float clamp;          // sum of the negative depths reset to zero
    float drn_s, drn_c;   // drained depth (land cover; Kahan pair)
};

__device__ __forceinline__ void m_load4(float (&v)[4], const float* p)
{
    float4 t = ldg4(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void m_store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// The links of one row of a lane's four cells: east links (Eq. 2-3, or the
// free-outflow edge) and south links.  INTERIOR: all four cells and their
// east neighbours lie inside the grid, so no per-cell edge tests are needed.
template <bool INTERIOR, int LIM = -1>
__device__ __forceinline__ void row_links(const float (&hC)[4], const float (&zC)[4],
                                          const float (&nC)[4], const float (&hS)[4],
                                          const float (&zS)[4], const float (&nS)[4],
                                          const float (&qxo)[4], const float (&qyo)[4], float hE,
                                          float zE, float nE, bool has_s, int c, int nx, float s,
                                          float s_half, const FaceK& k, int east_out,
                                          int south_out, float (&qxE)[4], float (&qyS)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int cj = c + j;
        const float h2 = (j < 3) ? hC[j + 1] : hE;
        const float z2 = (j < 3) ? zC[j + 1] : zE;
        const float n2 = (j < 3) ? nC[j + 1] : nE;
        float q;
        if (INTERIOR || cj < nx - 1)
            q = link_q<LIM>(hC[j], zC[j], h2, z2, qxo[j], __fmul_rn(s_half, __fadd_rn(nC[j], n2)), k);
        else if (cj == nx - 1)
            q = east_out ? outflow_q<LIM>(hC[j], qxo[j], __fmul_rn(s, nC[j]), k) : 0.0f;
        else
            q = 0.0f;
        qxE[j] = q;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float q = 0.0f;
        if (INTERIOR || c + j < nx) {
            if (has_s)
                q = link_q<LIM>(hC[j], zC[j], hS[j], zS[j], qyo[j],
                           __fmul_rn(s_half, __fadd_rn(nC[j], nS[j])), k);
            else if (south_out)
                q = outflow_q<LIM>(hC[j], qyo[j], __fmul_rn(s, nC[j]), k);
        }
        qyS[j] = q;
    }
}

// Continuity (Eq. 5 -> Eq. 1) with rain and the wet/dry clamp for a lane's
// four cells.  Clamped cells keep a negative zero: the adjoint reads the sign
// bit to know that branch was taken (and so do cells that land-cover
// drainage emptied).  LC (land cover, Section 4.1): the rain
// that stays depends on the cell's class, and the class's drainage then
// removes at most the water present.
template <bool INTERIOR, bool LC = false>
__device__ __forceinline__ void row_depths(const float (&hC)[4], const float (&qxE)[4],
                                           const float (&qyN)[4], const float (&qyS)[4], float qW0,
                                           int c, int nx, float dt_dx, float dr, float& clamp,
                                           float& hmax, float (&hN)[4],
                                           const float* drv = nullptr, const float* ddv = nullptr,
                                           float* drn_s = nullptr, float* drn_c = nullptr)
{
    float row_sink = 0.0f;  // LC: the row's drained depth, compensated once per row
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float hn = 0.0f;
        if (INTERIOR || c + j < nx) {
            const float qW = (j == 0) ? qW0 : qxE[j - 1];
            const float net = __fadd_rn(__fsub_rn(qW, qxE[j]), __fsub_rn(qyN[j], qyS[j]));
            // the step's increment (fluxes and rain) is formed first and
            // added to the depth once: adding the same rain depth to every
            // cell on its own rounds every cell of a binade the same way,
            // a bias that builds up in the stored volume
            if (LC) {
                const float hp = __fadd_rn(hC[j], __fmaf_rn(dt_dx, net, drv[j]));
                const float sink = fminf(ddv[j], fmaxf(hp, 0.0f));
                hn = __fsub_rn(hp, sink);
                // drainage that took all the water present leaves a depth
                // that does not depend on the one before: marked like a
                // clamped cell
                if (hp > 0.0f && sink == hp) hn = -0.0f;
                row_sink = __fadd_rn(row_sink, sink);
            } else {
                hn = __fadd_rn(hC[j], __fmaf_rn(dt_dx, net, dr));
            }
            if (hn < 0.0f) {
                clamp = __fsub_rn(clamp, hn);
                hn = -0.0f;
            }
            hmax = fmax_nan(hmax, hn);  // a NaN anywhere stays in the maximum
        }
        hN[j] = hn;
    }
    if (LC) kahan_add(*drn_s, *drn_c, row_sink);
}

template <bool LC = false>
__device__ __forceinline__ MarchOut march_rows(const float* __restrict__ src, float* __restrict__ dst,
                                               float* ck, float* hm, const float* __restrict__ z,
                                               const float* __restrict__ n, size_t plane, int ny,
                                               int nx, int ld, int c0, int r0, int r1, int lane,
                                               const FaceK& k, float dt_dx, float s, float dr,
                                               int east_out, int south_out,
                                               const LandK* lk = nullptr)
{
    const float s_half = 0.5f * s;
    const float* __restrict__ sh = src;
    const float* __restrict__ sqx = src + plane;
    const float* __restrict__ sqy = src + 2 * plane;
    float* __restrict__ dh = dst;
    float* __restrict__ dqx = dst + plane;
    float* __restrict__ dqy = dst + 2 * plane;

    const int c = c0 + 4 * lane;
    const bool act = c < nx;           // lane owns at least one real cell
    const bool east_halo = (lane == 31) && (c + 4 < nx);
    const bool interior = (c + 4 < nx);  // all four cells and their east neighbours inside

    float hC[4] = {0, 0, 0, 0}, zC[4] = {0, 0, 0, 0}, nC[4] = {0, 0, 0, 0};
    float qyN[4] = {0, 0, 0, 0};
    uint32_t clsC = 0;  // land classes of the lane's four cells in the current row
    // classes of the cells just east and west of the span (current row, and
    // the next row's loaded one iteration ahead)
    uint32_t eC = 0, wC = 0, eN = 0, wN = 0;
    if (LC) {
        if (c0 + 128 < nx) eC = lk->cls[(size_t)r0 * ld + c0 + 128];
        if (c0 > 0) wC = lk->cls[(size_t)r0 * ld + c0 - 1];
    }
    // land classes (LC): looked up by the whole warp (shuffles), outside
    // any lane-dependent branch
    uint32_t clsU = 0;
    if (LC) {
        if (act) {
            clsC = cls_word(lk->cls, (size_t)r0 * ld + c);
            if (r0 > 0) clsU = cls_word(lk->cls, (size_t)(r0 - 1) * ld + c);
        }
        land_n4(nC, clsC, *lk);
    }
    float nUl[4] = {0, 0, 0, 0};
    if (LC && r0 > 0) land_n4(nUl, clsU, *lk);
    if (act) {
        const size_t o = (size_t)r0 * ld + c;
        m_load4(hC, sh + o);
        m_load4(zC, z + o);
        if (!LC) m_load4(nC, n + o);
        if (r0 > 0) {
            float hU[4], zU[4], nU[4], qU[4];
            const size_t ou = o - ld;
            m_load4(hU, sh + ou);
            m_load4(zU, z + ou);
            if (LC) {
#pragma unroll
                for (int j = 0; j < 4; ++j) nU[j] = nUl[j];
            } else {
                m_load4(nU, n + ou);
            }
            m_load4(qU, sqy + ou);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                qyN[j] = (c + j < nx)
                             ? link_q(hU[j], zU[j], hC[j], zC[j], qU[j],
                                      __fmul_rn(s_half, __fadd_rn(nU[j], nC[j])), k)
                             : 0.0f;
        }
    }

    float hmax = 0.0f;
    float out_s = 0.0f, out_c = 0.0f, clamp = 0.0f, drn_s = 0.0f, drn_c = 0.0f;

#pragma unroll 2
    for (int r = r0; r < r1; ++r) {
        const size_t o = (size_t)r * ld + c;
        const bool has_s = (r + 1 < ny);
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0};
        float qxo[4] = {0, 0, 0, 0}, qyo[4] = {0, 0, 0, 0};
        uint32_t clsS = 0;
        if (LC && has_s) {
            const size_t rs = (size_t)(r + 1) * ld;
            if (c0 + 128 < nx) eN = lk->cls[rs + c0 + 128];
            if (c0 > 0) wN = lk->cls[rs + c0 - 1];
        }
        if (act) {
            if (has_s) {
                m_load4(hS, sh + o + ld);
                m_load4(zS, z + o + ld);
                if (LC)
                    clsS = cls_word(lk->cls, o + ld);
                else
                    m_load4(nS, n + o + ld);
            }
            m_load4(qxo, sqx + o);
            m_load4(qyo, sqy + o);
        }
        float nEl = 0.0f, nWl = 0.0f, drv[4], ddv[4];
        if (LC) {
            if (has_s) land_n4(nS, clsS, *lk);
            nEl = land_get(lk->n, eC);
            nWl = land_get(lk->n, wC);
            land_src4(drv, ddv, clsC, *lk);
        }
        // east neighbour of the lane's last cell: next lane's first cell
        float hE = __shfl_down_sync(0xffffffffu, hC[0], 1);
        float zE = __shfl_down_sync(0xffffffffu, zC[0], 1);
        float nE = __shfl_down_sync(0xffffffffu, nC[0], 1);
        if (east_halo) {
            const size_t oe = (size_t)r * ld + c + 4;
            hE = __ldg(sh + oe);
            zE = __ldg(z + oe);
            nE = LC ? nEl : __ldg(n + oe);
        }
        float qxE[4], qyS[4];
        if (interior)
            row_links<true>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                            east_out, south_out, qxE, qyS);
        else
            row_links<false>(hC, zC, nC, hS, zS, nS, qxo, qyo, hE, zE, nE, has_s, c, nx, s, s_half, k,
                             east_out, south_out, qxE, qyS);
        // west link of the lane's first cell: previous lane's last east link
        float qW0 = __shfl_up_sync(0xffffffffu, qxE[3], 1);
        if (lane == 0) {
            qW0 = (r >= k.in_r0 && r < k.in_r1) ? k.q_in : 0.0f;  // west edge: wall or inflow
            if (c0 > 0) {  // recompute the neighbouring span's link (halo)
                const size_t ow = (size_t)r * ld + c0 - 1;
                const float nw = LC ? nWl : __ldg(n + ow);
                qW0 = link_q(__ldg(sh + ow), __ldg(z + ow), hC[0], zC[0], __ldg(sqx + ow),
                             __fmul_rn(s_half, __fadd_rn(nw, nC[0])), k);
            }
        }
        float hN[4];
        if (interior)
            row_depths<true, LC>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hN,
                                 drv, ddv, &drn_s, &drn_c);
        else
            row_depths<false, LC>(hC, qxE, qyN, qyS, qW0, c, nx, dt_dx, dr, clamp, hmax, hN,
                                  drv, ddv, &drn_s, &drn_c);
        // links leaving the domain this row: the east edge link (one lane)
        // and, on the last row, the south edge links
        float ev = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c + j == nx - 1 && east_out) ev = qxE[j];
        if (!has_s && south_out)
            ev = __fadd_rn(ev, __fadd_rn(__fadd_rn(qyS[0], qyS[1]), __fadd_rn(qyS[2], qyS[3])));
        kahan_add(out_s, out_c, ev);
        if (act) {
            m_store4(dh + o, hN);
            m_store4(dqx + o, qxE);
            m_store4(dqy + o, qyS);
            if (ck) {
                m_store4(ck + o, hN);
                m_store4(ck + plane + o, qxE);
                m_store4(ck + 2 * plane + o, qyS);
            }
            if (hm) {  // loaded here, not ahead: registers are scarce in this kernel
                const float4 hmo = *reinterpret_cast<const float4*>(hm + o);
                *reinterpret_cast<float4*>(hm + o) =
                    make_float4(fmaxf(hmo.x, hN[0]), fmaxf(hmo.y, hN[1]), fmaxf(hmo.z, hN[2]),
                                fmaxf(hmo.w, hN[3]));
            }
        }
        // march: this row's south links are the next row's north links
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            qyN[j] = qyS[j];
            hC[j] = hS[j];
            zC[j] = zS[j];
            nC[j] = nS[j];
        }
        clsC = clsS;
        eC = eN;
        wC = wN;
    }

    MarchOut out;
    out.hmax = hmax;
    out.bad = !(hmax <= 3.0e38f);  // a NaN or an overflow anywhere
    out.out_s = out_s;
    out.out_c = out_c;
    out.clamp = clamp;
    out.drn_s = drn_s;
    out.drn_c = drn_c;
    return out;
}

}  // namespace flood
