// Per-row arithmetic of the reverse stencil, shared by the direct-load
// (adjoint_kernel.cu) and TMA-staged (adjoint_tma.cu) adjoint kernels so the
// two give bit-identical gradients.  The caller supplies the values of a
// lane's four cells from wherever it staged them.
//
// Straight-line code: every link's partials are computed in full and the
// branch the forward step took (dry link, limiter, outflow clip) is applied
// by selection, so rows that mix wet and dry links cost the warp no
// divergent paths.  The roughness enters Eq. 2 only through n_link^2, so
// n_link dq'/dn_link = -2 q' fric / D needs no division by n_link, and
// dq'/dq is formed from b h^(-7/3) rather than by dividing by q.
#pragma once

#include "flood_internal.cuh"

namespace flood {

// Partials of one new link flux q' (Eq. 2-3 and the limiter): with respect
// to the depths of its two cells and its old flux, and g2 = n_link dq'/dn_link.
struct LinkD {
    float dh1, dh2, dq, g2;
};

// Interior link (same forward arithmetic and branch decisions as link_q).
template <int LIM>
__device__ __forceinline__ LinkD link_d(float h1, float z1, float h2, float z2, float q, float nl,
                                        const FaceK& k)
{
    // the forward quantities, rounded exactly as link_q rounds them
    const float dz = __fsub_rn(z2, z1);
    const float a1 = __fsub_rn(h1, fmaxf(dz, 0.0f));
    const float a2 = __fadd_rn(h2, fminf(dz, 0.0f));
    const float hf = fmaxf(a1, a2);
    const float dS = __fadd_rn(dz, __fsub_rn(h2, h1));
    const float num = __fmaf_rn(-__fmul_rn(k.gdt_dx, hf), dS, q);
    const float b = __fmul_rn(k.gdt, __fmul_rn(nl, nl));
    const float ih = inv_h73(hf);
    const float fric = __fmul_rn(__fmul_rn(b, fabsf(q)), ih);
    const float invD = rcp_approx(__fadd_rn(1.0f, fric));
    const float qs = __fmul_rn(num, invD);
    // dq'/dhf = -G dS / D + (7/3) q' fric / (D hf);  dq'/d(dx S) = -G hf / D
    // dq'/dq = (1 - q' b h^(-7/3) sgn q) / D;        n dq'/dn = -2 q' fric / D
    const float u = qs * invD;
    const float qt = u * fric;
    const float dq_dS = -(k.gdt_dx * hf) * invD;
    const float dq_dhf = __fmaf_rn(-(k.gdt_dx * dS), invD, 2.33333333f * qt * rcp_approx(hf));
    const bool first = a1 >= a2;  // Eq. 3's tie goes to the first argument
    const float dh1 = (first ? dq_dhf : 0.0f) - dq_dS;
    const float dh2 = (first ? 0.0f : dq_dhf) + dq_dS;
    const float ub = u * (b * ih);
    const float dq = invD - (q > 0.0f ? ub : (q < 0.0f ? -ub : 0.0f));
    bool hi = false, lo = false;
    if (LIM) {
        hi = qs > __fmul_rn(h1, k.dx_4dt);
        lo = qs < -__fmul_rn(h2, k.dx_4dt);
    }
    const bool wet = hf > k.h_eps;
    const bool fr = wet && !(hi || lo);
    LinkD r;
    r.dh1 = fr ? dh1 : ((wet && hi) ? k.dx_4dt : 0.0f);
    r.dh2 = fr ? dh2 : ((wet && lo) ? -k.dx_4dt : 0.0f);
    r.dq = fr ? dq : 0.0f;
    r.g2 = fr ? -2.0f * qt : 0.0f;
    return r;
}

// Free-outflow link (ghost with the edge depth, as outflow_q): dh1 is the
// total derivative with respect to the edge cell's depth.
template <int LIM>
__device__ __forceinline__ LinkD outflow_d(float h, float q, float nl, const FaceK& k)
{
    const float num = __fmaf_rn(-__fmul_rn(k.gdt_dx, h), -k.edge_drop, q);
    const float b = __fmul_rn(k.gdt, __fmul_rn(nl, nl));
    const float ih = inv_h73(h);
    const float fric = __fmul_rn(__fmul_rn(b, fabsf(q)), ih);
    const float invD = rcp_approx(__fadd_rn(1.0f, fric));
    const float qs = __fmul_rn(num, invD);
    const float u = qs * invD;
    const float qt = u * fric;
    const float dh = __fmaf_rn(k.gdt_dx * k.edge_drop, invD, 2.33333333f * qt * rcp_approx(h));
    const float ub = u * (b * ih);
    const float dq = invD - (q > 0.0f ? ub : (q < 0.0f ? -ub : 0.0f));
    const bool hi = LIM && qs > __fmul_rn(h, k.dx_4dt);
    const bool wet = h > k.h_eps;
    const bool fr = wet && !hi && qs > 0.0f;  // only outward flow passes
    LinkD r;
    r.dh1 = fr ? dh : ((wet && hi) ? k.dx_4dt : 0.0f);
    r.dh2 = 0.0f;
    r.dq = fr ? dq : 0.0f;
    r.g2 = fr ? -2.0f * qt : 0.0f;
    return r;
}

// 1 / (sum of the roughness values a link's n_link is made of); a zero sum
// (no friction, so g2 = 0) gives a finite factor and a zero weight.
__device__ __forceinline__ float inv_nsum(float ns) { return rcp_approx(fmaxf(ns, 1.0e-30f)); }

__device__ __forceinline__ float masked(float h_after, float lam)
{
    return signbit(h_after) ? 0.0f : lam;  // clamped cells pass no sensitivity
}

// The strip's north links (the row above the strip's first row), recomputed:
// their contributions to the first row's depth and Manning sensitivities.
template <int LIM>
__device__ __forceinline__ void north_carry(const float (&hU)[4], const float (&zU)[4],
                                            const float (&nU)[4], const float (&qU)[4],
                                            const float (&lqU)[4], const float (&lU)[4],
                                            const float (&hC)[4], const float (&zC)[4],
                                            const float (&nC)[4], const float (&lC)[4], int c,
                                            int nx, float s_half, float T, const FaceK& k,
                                            float (&carH)[4], float (&carN)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (c + q >= nx) continue;
        const float ns = __fadd_rn(nU[q], nC[q]);
        const LinkD d = link_d<LIM>(hU[q], zU[q], hC[q], zC[q], qU[q], __fmul_rn(s_half, ns), k);
        const float mu = lqU[q] + T * (lC[q] - lU[q]);
        carH[q] = mu * d.dh2;
        carN[q] = (mu * d.g2) * inv_nsum(ns);
    }
}

// West neighbour of the span's first cell (lane 0 only): state before the
// step, lambda of its east link, masked depth lambda.
struct WestIn {
    float h, z, n, qx, lqx, l;
};

// One row of the reverse stencil for a lane's four cells.  C: this row, S:
// the row below (zeros past the last row), E: the next lane's first cell
// (the tile's halo for the last lane).  Writes the sensitivities to the
// step's inputs (lh, lx, ly) and the Manning contribution (gnr), updates the
// north-link carries, and adds this row's rain partial (sum of lambda~) and
// scale partial (sum of mu n dq'/dn over the lane's links, to be divided by
// the scale) to gr_row and gs_row.  INTERIOR: the span lies wholly inside the
// grid with an interior link east of its last cell (c0 + 128 < nx).  RW: the
// rain partial weighs each cell by rw, the fraction of the rain that stays
// on it (land cover, Section 4.1).
template <bool INTERIOR, int LIM, bool RW = false>
__device__ __forceinline__ void adjoint_row(
    const float (&hC)[4], const float (&zC)[4], const float (&nC)[4], const float (&lC)[4],
    const float (&hS)[4], const float (&zS)[4], const float (&nS)[4], const float (&lS)[4],
    const float (&qxo)[4], const float (&qyo)[4], const float (&lqx)[4], const float (&lqy)[4],
    float hE, float zE, float nE, float lE, bool west_halo, const WestIn& wi, bool has_s, int c,
    int nx, int lane, float s, float s_half, float T, const FaceK& k, int east_out,
    int south_out, float (&carH)[4], float (&carN)[4], float& gr_row, float& gs_row,
    float (&lh)[4], float (&lx)[4], float (&ly)[4], float (&gnr)[4], const float* rw = nullptr)
{
    const LinkD zero{0.0f, 0.0f, 0.0f, 0.0f};
    // east links: mu = lambda_q' + T (lambda~_east - lambda~_here); per link
    // mu dq'/dh1 (this cell), mu dq'/dh2 (the east cell), mu dq'/dq, and the
    // Manning weight mu n dq'/dn / (sum of the n it is made of)
    float pE1[4], pE2[4], xE[4], wE[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int cj = c + q;
        const float h2 = (q < 3) ? hC[q + 1] : hE;
        const float z2 = (q < 3) ? zC[q + 1] : zE;
        const float n2 = (q < 3) ? nC[q + 1] : nE;
        const float l2 = (q < 3) ? lC[q + 1] : lE;
        LinkD d = zero;
        float mu = 0.0f, w = 0.0f;
        if (INTERIOR || cj < nx - 1) {
            const float ns = __fadd_rn(nC[q], n2);
            d = link_d<LIM>(hC[q], zC[q], h2, z2, qxo[q], __fmul_rn(s_half, ns), k);
            mu = lqx[q] + T * (l2 - lC[q]);
            w = inv_nsum(ns);
        } else if (cj == nx - 1) {
            if (east_out) d = outflow_d<LIM>(hC[q], qxo[q], __fmul_rn(s, nC[q]), k);
            mu = lqx[q] - T * lC[q];
            w = inv_nsum(nC[q]);
        }
        const float G = mu * d.g2;
        gs_row += G;
        pE1[q] = mu * d.dh1;
        pE2[q] = mu * d.dh2;
        xE[q] = mu * d.dq;
        wE[q] = G * w;
    }
    // west link of the lane's first cell
    float pW2 = __shfl_up_sync(0xffffffffu, pE2[3], 1);
    float wW = __shfl_up_sync(0xffffffffu, wE[3], 1);
    if (lane == 0) {
        pW2 = 0.0f;
        wW = 0.0f;
        if (west_halo) {
            const float ns = __fadd_rn(wi.n, nC[0]);
            const LinkD d = link_d<LIM>(wi.h, wi.z, hC[0], zC[0], wi.qx, __fmul_rn(s_half, ns), k);
            const float mu = wi.lqx + T * (lC[0] - wi.l);
            pW2 = mu * d.dh2;
            wW = (mu * d.g2) * inv_nsum(ns);
        }
    }
    // south links
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int cj = c + q;
        const bool in = INTERIOR || cj < nx;
        LinkD d = zero;
        float mu = 0.0f, w = 0.0f;
        if (in) {
            if (has_s) {
                const float ns = __fadd_rn(nC[q], nS[q]);
                d = link_d<LIM>(hC[q], zC[q], hS[q], zS[q], qyo[q], __fmul_rn(s_half, ns), k);
                mu = lqy[q] + T * (lS[q] - lC[q]);
                w = inv_nsum(ns);
            } else {
                if (south_out) d = outflow_d<LIM>(hC[q], qyo[q], __fmul_rn(s, nC[q]), k);
                mu = lqy[q] - T * lC[q];
                w = inv_nsum(nC[q]);
            }
            gr_row = RW ? __fmaf_rn(lC[q], rw[q], gr_row) : gr_row + lC[q];
        }
        const float G = mu * d.g2;
        gs_row += G;
        const float wS = G * w;
        const float pw2 = (q == 0) ? pW2 : pE2[q - 1];
        const float ww = (q == 0) ? wW : wE[q - 1];
        lh[q] = in ? lC[q] + pE1[q] + pw2 + mu * d.dh1 + carH[q] : 0.0f;
        lx[q] = in ? xE[q] : 0.0f;
        ly[q] = in ? mu * d.dq : 0.0f;
        gnr[q] = in ? wE[q] + ww + wS + carN[q] : 0.0f;
        carH[q] = mu * d.dh2;
        carN[q] = wS;
    }
}

// Land cover: the warp's drainage partial (sum over the cells that drainage
// left wet of lambda~), widened to FP64 and summed over lanes, times -dt
// (dL/d(drainage rate)), added to the warp's slot.
__device__ __forceinline__ void adjoint_drain_partial(double* gdpart, int nslot, int m, int slot,
                                                      int lane, float gd_s, float gd_c, double dt)
{
    double g = ((double)gd_s - (double)gd_c) * -dt;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) g += __shfl_xor_sync(0xffffffffu, g, off);
    if (lane == 0) gdpart[(size_t)m * nslot + slot] += g;
}

// The drainage partial of a lane's four cells in one row: lambda~ of the
// cells of a draining class (df = 1) that the step left wet.
__device__ __forceinline__ float drain_row(const float (&lC)[4], const float (&ha)[4],
                                           const float (&df)[4])
{
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) acc += ha[q] > 0.0f ? lC[q] * df[q] : 0.0f;
    return acc;
}

// The warp's rain and scale partials, widened to FP64, summed over lanes
// and added to the warp's slot (one slot per span and strip).  rdt: the
// step's rain depth per unit multiplier; rs: 1 / scale.
__device__ __forceinline__ void adjoint_partials(double* gpart, int nslot, int m, int slot,
                                                 int lane, float gr_s, float gr_c, float gs_s,
                                                 float gs_c, double rdt, double rs)
{
    double g_rain = ((double)gr_s - (double)gr_c) * rdt;
    double g_scale = ((double)gs_s - (double)gs_c) * rs;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        g_rain += __shfl_xor_sync(0xffffffffu, g_rain, off);
        g_scale += __shfl_xor_sync(0xffffffffu, g_scale, off);
    }
    if (lane == 0) {
        double* v = gpart + ((size_t)m * nslot + slot) * 2;
        v[0] += g_rain;
        v[1] += g_scale;
    }
}

}  // namespace flood
