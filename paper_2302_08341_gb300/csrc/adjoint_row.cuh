// Per-row arithmetic of the reverse stencil, shared by the direct-load
// (adjoint_kernel.cu) and TMA-staged (adjoint_tma.cu) adjoint kernels so the
// two give bit-identical gradients.  The caller supplies the values of a
// lane's four cells from wherever it staged them.
#pragma once

#include "flood_internal.cuh"

namespace flood {

struct LinkD {
    float dh1, dh2, dq, dnl;  // partials of the new link flux
};

// Partials of the interior link flux (same arithmetic and branch decisions
// as link_q in the forward kernel).
__device__ __forceinline__ LinkD link_d(float h1, float z1, float h2, float z2, float q, float nl,
                                        const FaceK& k, float L)
{
    LinkD r{0.0f, 0.0f, 0.0f, 0.0f};
    const float dz = __fsub_rn(z2, z1);
    const float a1 = __fsub_rn(h1, fmaxf(dz, 0.0f));
    const float a2 = __fadd_rn(h2, fminf(dz, 0.0f));
    const float hf = fmaxf(a1, a2);
    if (!(hf > k.h_eps)) return r;
    const bool first = a1 >= a2;
    const float dS = __fadd_rn(dz, __fsub_rn(h2, h1));
    const float num = __fmaf_rn(-__fmul_rn(k.gdt_dx, hf), dS, q);
    const float c = __fmul_rn(__fmul_rn(k.gdt, __fmul_rn(nl, nl)), fabsf(q));
    const float fric = __fmul_rn(c, inv_h73(hf));
    const float D = __fadd_rn(1.0f, fric);
    const float invD = rcp_approx(D);
    const float qs = __fmul_rn(num, invD);
    if (k.limiter) {
        const float lim = __fmul_rn(qs > 0.0f ? h1 : h2, k.dx_4dt);
        if (qs > lim) { r.dh1 = L; return r; }
        if (qs < -lim) { r.dh2 = -L; return r; }
    }
    const float t = __fmul_rn(fric, invD);                      // fric / D in [0, 1)
    // dq'/dhf = -G dS / D + (7/3) q' t / hf ; dq'/d(dx S) = -G hf / D
    const float dq_dhf = __fmaf_rn(-k.gdt_dx * dS, invD, 2.33333333f * __fdividef(qs * t, hf));
    const float dq_dS = -k.gdt_dx * hf * invD;
    r.dh1 = (first ? dq_dhf : 0.0f) - dq_dS;
    r.dh2 = (first ? 0.0f : dq_dhf) + dq_dS;
    r.dq = invD - (q == 0.0f ? 0.0f : __fdividef(qs * t, q));
    r.dnl = nl > 0.0f ? -2.0f * __fdividef(qs * t, nl) : 0.0f;
    return r;
}

// Partials of the free-outflow link (ghost with the edge depth): dh is the
// total derivative with respect to the edge cell's depth.
__device__ __forceinline__ LinkD outflow_d(float h, float q, float ncell, const FaceK& k, float L)
{
    LinkD r{0.0f, 0.0f, 0.0f, 0.0f};
    if (!(h > k.h_eps)) return r;
    const float num = __fmaf_rn(-__fmul_rn(k.gdt_dx, h), -k.edge_drop, q);
    const float c = __fmul_rn(__fmul_rn(k.gdt, __fmul_rn(ncell, ncell)), fabsf(q));
    const float fric = __fmul_rn(c, inv_h73(h));
    const float D = __fadd_rn(1.0f, fric);
    const float invD = rcp_approx(D);
    const float qs = __fmul_rn(num, invD);
    if (k.limiter && qs > __fmul_rn(h, k.dx_4dt)) { r.dh1 = L; return r; }
    if (!(qs > 0.0f)) return r;
    const float t = __fmul_rn(fric, invD);
    r.dh1 = __fmaf_rn(k.gdt_dx * k.edge_drop, invD, 2.33333333f * __fdividef(qs * t, h));
    r.dq = invD - (q == 0.0f ? 0.0f : __fdividef(qs * t, q));
    r.dnl = ncell > 0.0f ? -2.0f * __fdividef(qs * t, ncell) : 0.0f;
    return r;
}

__device__ __forceinline__ float masked(float h_after, float lam)
{
    return signbit(h_after) ? 0.0f : lam;  // clamped cells pass no sensitivity
}

// The strip's north links (the row above the strip's first row), recomputed:
// their contributions to the first row's depth and Manning sensitivities.
__device__ __forceinline__ void north_carry(const float (&hU)[4], const float (&zU)[4],
                                            const float (&nU)[4], const float (&qU)[4],
                                            const float (&lqU)[4], const float (&lU)[4],
                                            const float (&hC)[4], const float (&zC)[4],
                                            const float (&nC)[4], const float (&lC)[4], int c,
                                            int nx, float s_half, float T, float L,
                                            const FaceK& k, float (&carH)[4], float (&carN)[4])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (c + q >= nx) continue;
        const LinkD d = link_d(hU[q], zU[q], hC[q], zC[q], qU[q],
                               __fmul_rn(s_half, __fadd_rn(nU[q], nC[q])), k, L);
        const float mu = lqU[q] + T * (lC[q] - lU[q]);
        carH[q] = mu * d.dh2;
        carN[q] = mu * d.dnl * s_half;
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
// north-link carries and the compensated rain / scale partials.
__device__ __forceinline__ void adjoint_row(
    const float (&hC)[4], const float (&zC)[4], const float (&nC)[4], const float (&lC)[4],
    const float (&hS)[4], const float (&zS)[4], const float (&nS)[4], const float (&lS)[4],
    const float (&qxo)[4], const float (&qyo)[4], const float (&lqx)[4], const float (&lqy)[4],
    float hE, float zE, float nE, float lE, bool west_halo, const WestIn& wi, bool has_s, int c,
    int nx, int lane, float s, float s_half, float T, float L, const FaceK& k, int east_out,
    int south_out, float (&carH)[4], float (&carN)[4], float& gr_s, float& gr_c, float& gs_s,
    float& gs_c, float (&lh)[4], float (&lx)[4], float (&ly)[4], float (&gnr)[4])
{
    // east links: mu = lambda_q' + T (lambda~_east - lambda~_here)
    float muE[4], dEh1[4], dEh2[4], dEq[4], dEn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int cj = c + q;
        const float h2 = (q < 3) ? hC[q + 1] : hE;
        const float z2 = (q < 3) ? zC[q + 1] : zE;
        const float n2 = (q < 3) ? nC[q + 1] : nE;
        const float l2 = (q < 3) ? lC[q + 1] : lE;
        LinkD d{0.0f, 0.0f, 0.0f, 0.0f};
        float mu = 0.0f, nl_w = 0.0f;
        if (cj < nx - 1) {
            d = link_d(hC[q], zC[q], h2, z2, qxo[q], __fmul_rn(s_half, __fadd_rn(nC[q], n2)), k, L);
            mu = lqx[q] + T * (l2 - lC[q]);
            nl_w = 0.5f * (nC[q] + n2);
            dEn[q] = d.dnl * s_half;
        } else if (cj == nx - 1) {
            if (east_out) d = outflow_d(hC[q], qxo[q], __fmul_rn(s, nC[q]), k, L);
            mu = lqx[q] - T * lC[q];
            nl_w = nC[q];
            dEn[q] = d.dnl * s;
        } else {
            dEn[q] = 0.0f;
        }
        muE[q] = mu; dEh1[q] = d.dh1; dEh2[q] = d.dh2; dEq[q] = d.dq;
        kahan_add(gs_s, gs_c, mu * d.dnl * nl_w);
    }
    // west link of the lane's first cell
    float muW = __shfl_up_sync(0xffffffffu, muE[3], 1);
    float dWh2 = __shfl_up_sync(0xffffffffu, dEh2[3], 1);
    float dWn = __shfl_up_sync(0xffffffffu, dEn[3], 1);
    if (lane == 0) {
        muW = 0.0f; dWh2 = 0.0f; dWn = 0.0f;
        if (west_halo) {
            const LinkD d = link_d(wi.h, wi.z, hC[0], zC[0], wi.qx,
                                   __fmul_rn(s_half, __fadd_rn(wi.n, nC[0])), k, L);
            muW = wi.lqx + T * (lC[0] - wi.l);
            dWh2 = d.dh2;
            dWn = d.dnl * s_half;
        }
    }
    // south links
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int cj = c + q;
        LinkD d{0.0f, 0.0f, 0.0f, 0.0f};
        float mu = 0.0f, dn = 0.0f, nl_w = 0.0f;
        if (cj < nx) {
            if (has_s) {
                d = link_d(hC[q], zC[q], hS[q], zS[q], qyo[q],
                           __fmul_rn(s_half, __fadd_rn(nC[q], nS[q])), k, L);
                mu = lqy[q] + T * (lS[q] - lC[q]);
                dn = d.dnl * s_half;
                nl_w = 0.5f * (nC[q] + nS[q]);
            } else {
                if (south_out) d = outflow_d(hC[q], qyo[q], __fmul_rn(s, nC[q]), k, L);
                mu = lqy[q] - T * lC[q];
                dn = d.dnl * s;
                nl_w = nC[q];
            }
            kahan_add(gs_s, gs_c, mu * d.dnl * nl_w);
            kahan_add(gr_s, gr_c, lC[q]);
        }
        const float muw = (q == 0) ? muW : muE[q - 1];
        const float dwh = (q == 0) ? dWh2 : dEh2[q - 1];
        const float dwn = (q == 0) ? dWn : dEn[q - 1];
        const bool in = cj < nx;
        lh[q] = in ? lC[q] + muE[q] * dEh1[q] + muw * dwh + mu * d.dh1 + carH[q] : 0.0f;
        lx[q] = in ? muE[q] * dEq[q] : 0.0f;
        ly[q] = in ? mu * d.dq : 0.0f;
        gnr[q] = in ? muE[q] * dEn[q] + muw * dwn + mu * dn + carN[q] : 0.0f;
        carH[q] = mu * d.dh2;
        carN[q] = mu * dn;
    }
}

// The warp's rain and scale partials, widened to FP64, summed over lanes
// and added to the warp's slot (one slot per span and strip).
__device__ __forceinline__ void adjoint_partials(double* gpart, int nslot, int m, int slot,
                                                 int lane, float gr_s, float gr_c, float gs_s,
                                                 float gs_c, double rdt)
{
    double g_rain = ((double)gr_s - (double)gr_c) * rdt;
    double g_scale = (double)gs_s - (double)gs_c;
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
