// Reverse mode of the fused local-inertial step (extension beyond the
// paper): given the loss's sensitivities to the state after step j
// (lambda_{j+1} = dL/d(h, qx, qy)), produce those to the state before it
// (lambda_j) and accumulate dL/dn (per cell, per member), dL/d(rain
// multiplier) and dL/d(Manning scale).  The step length is held fixed (the
// recorded schedule); at every kink (Eq. 3's max, the limiter, the wet/dry
// test, the outflow clip, the negative-depth clamp) the derivative of the
// branch taken is used, ties in Eq. 3 going to the first argument.  A cell
// whose depth was clamped carries a negative zero in the recorded state,
// which is how this kernel knows that branch was taken.
//
// Layout and traversal mirror the forward kernel: a warp owns 128 columns
// (float4 per lane) of a strip of rows of one member and marches down; the
// west link comes from the neighbouring lane by shuffle (recomputed by lane 0
// at the span edge), the north link's contribution is carried from the row
// above (recomputed at the strip top).
//
// HBM traffic per member-cell-step: state before the step (12 B), depth after
// it (4 B), lambda in (12 B), lambda out (12 B), per-cell Manning gradient
// read + write (8 B), z and n shared per tile.
#include "adjoint.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;

struct LinkD {
    float dh1, dh2, dq, dnl;  // partials of the new link flux
};

__device__ __forceinline__ void load4(float (&v)[4], const float* p)
{
    float4 t = ldg4(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

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

template <int WM, int WC>
__global__ void __launch_bounds__(32 * WM * WC, 4) adjoint_kernel(const AdjArgs a)
{
    const int lane = threadIdx.x;
    const int wm = threadIdx.y % WM;
    const int wc = threadIdx.y / WM;
    const int m = blockIdx.x * WM + wm;
    const int span = blockIdx.y * WC + wc;
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;

    const int nx = a.nx, ny = a.ny, ld = a.ld;
    const size_t plane = a.plane, mstride = 3 * plane;
    const int c = c0 + 4 * lane;
    const bool act = c < nx;
    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, ny);
    const float* __restrict__ lin = a.lam + ((size_t)a.lam_in * a.M + m) * mstride;
    float* __restrict__ lout = a.lam + ((size_t)(1 - a.lam_in) * a.M + m) * mstride;

    const int j = a.seg_end[m] - 1 - a.rev_i;
    if (j < a.seg_first) {  // member idle in this launch: carry lambda over
        if (act)
            for (int r = r0; r < r1; ++r)
                for (int k = 0; k < 3; ++k) {
                    const size_t o = k * plane + (size_t)r * ld + c;
                    *reinterpret_cast<float4*>(lout + o) = ldg4(lin + o);
                }
        return;
    }
    const MemberPlan pl = a.log[(size_t)m * a.dt_log_cap + j];
    FaceK k;
    k.gdt_dx = pl.gdt_dx;
    k.gdt = pl.gdt;
    k.dx_4dt = pl.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    const float L = k.dx_4dt;
    const float T = pl.dt_dx;
    const float s = a.scale[m];
    const float s_half = 0.5f * s;

    const float* __restrict__ st = a.seg + ((size_t)(j - a.seg_first) * a.M + m) * mstride;
    const float* __restrict__ sh = st;
    const float* __restrict__ sqx = st + plane;
    const float* __restrict__ sqy = st + 2 * plane;
    const float* __restrict__ h1p = st + (size_t)a.M * mstride;  // depth after the step
    const float* __restrict__ z = a.z;
    const float* __restrict__ n = a.n;
    float* __restrict__ gn = a.gn ? a.gn + (size_t)m * plane : nullptr;
    const bool east_halo = (lane == 31) && (c + 4 < nx);

    float hC[4] = {0, 0, 0, 0}, zC[4] = {0, 0, 0, 0}, nC[4] = {0, 0, 0, 0}, lC[4] = {0, 0, 0, 0};
    float carH[4] = {0, 0, 0, 0}, carN[4] = {0, 0, 0, 0};  // north link: mu*dh2, mu*dnl
    if (act) {
        const size_t o = (size_t)r0 * ld + c;
        load4(hC, sh + o); load4(zC, z + o); load4(nC, n + o);
        float ha[4], la[4];
        load4(ha, h1p + o); load4(la, lin + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) lC[q] = masked(ha[q], la[q]);
        if (r0 > 0) {  // the strip's north links, recomputed
            const size_t u = o - ld;
            float hU[4], zU[4], nU[4], qU[4], lqU[4], haU[4], lhU[4];
            load4(hU, sh + u); load4(zU, z + u); load4(nU, n + u); load4(qU, sqy + u);
            load4(lqU, lin + 2 * plane + u); load4(haU, h1p + u); load4(lhU, lin + u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (c + q >= nx) continue;
                const LinkD d = link_d(hU[q], zU[q], hC[q], zC[q], qU[q],
                                       __fmul_rn(s_half, __fadd_rn(nU[q], nC[q])), k, L);
                const float mu = lqU[q] + T * (lC[q] - masked(haU[q], lhU[q]));
                carH[q] = mu * d.dh2;
                carN[q] = mu * d.dnl * s_half;
            }
        }
    }

    // FP32 compensated partials (sum of lambda~ for the rain gradient, of
    // mu * dq'/dn * n for the scale gradient), widened to FP64 once per warp
    float gr_s = 0.0f, gr_c = 0.0f, gs_s = 0.0f, gs_c = 0.0f;
    for (int r = r0; r < r1; ++r) {
        const size_t o = (size_t)r * ld + c;
        const bool has_s = (r + 1 < ny);
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0}, lS[4] = {0, 0, 0, 0};
        float qxo[4] = {0, 0, 0, 0}, qyo[4] = {0, 0, 0, 0}, lqx[4] = {0, 0, 0, 0}, lqy[4] = {0, 0, 0, 0};
        if (act) {
            if (has_s) {
                float ha[4], la[4];
                load4(hS, sh + o + ld); load4(zS, z + o + ld); load4(nS, n + o + ld);
                load4(ha, h1p + o + ld); load4(la, lin + o + ld);
#pragma unroll
                for (int q = 0; q < 4; ++q) lS[q] = masked(ha[q], la[q]);
            }
            load4(qxo, sqx + o); load4(qyo, sqy + o);
            load4(lqx, lin + plane + o); load4(lqy, lin + 2 * plane + o);
        }
        float hE = __shfl_down_sync(0xffffffffu, hC[0], 1);
        float zE = __shfl_down_sync(0xffffffffu, zC[0], 1);
        float nE = __shfl_down_sync(0xffffffffu, nC[0], 1);
        float lE = __shfl_down_sync(0xffffffffu, lC[0], 1);
        if (east_halo) {
            const size_t e = o + 4;
            hE = __ldg(sh + e); zE = __ldg(z + e); nE = __ldg(n + e);
            lE = masked(__ldg(h1p + e), __ldg(lin + e));
        }
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
                if (a.east_out) d = outflow_d(hC[q], qxo[q], __fmul_rn(s, nC[q]), k, L);
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
            if (c0 > 0) {
                const size_t w = o - 1;
                const float nw = __ldg(n + w);
                const LinkD d = link_d(__ldg(sh + w), __ldg(z + w), hC[0], zC[0], __ldg(sqx + w),
                                       __fmul_rn(s_half, __fadd_rn(nw, nC[0])), k, L);
                muW = __ldg(lin + plane + w) + T * (lC[0] - masked(__ldg(h1p + w), __ldg(lin + w)));
                dWh2 = d.dh2;
                dWn = d.dnl * s_half;
            }
        }
        // south links
        float lh[4], lx[4], ly[4], gnr[4];
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
                    if (a.south_out) d = outflow_d(hC[q], qyo[q], __fmul_rn(s, nC[q]), k, L);
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
        if (act) {
            store4(lout + o, lh);
            store4(lout + plane + o, lx);
            store4(lout + 2 * plane + o, ly);
            if (gn) {
                float4 g = *reinterpret_cast<const float4*>(gn + o);
                g.x += gnr[0]; g.y += gnr[1]; g.z += gnr[2]; g.w += gnr[3];
                *reinterpret_cast<float4*>(gn + o) = g;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            hC[q] = hS[q]; zC[q] = zS[q]; nC[q] = nS[q]; lC[q] = lS[q];
        }
    }
    double g_rain = ((double)gr_s - (double)gr_c) * pl.rdt;
    double g_scale = (double)gs_s - (double)gs_c;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        g_rain += __shfl_xor_sync(0xffffffffu, g_rain, off);
        g_scale += __shfl_xor_sync(0xffffffffu, g_scale, off);
    }
    if (lane == 0) {
        const int slot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
        double* v = a.gpart + ((size_t)m * a.nslot + slot) * 2;
        v[0] += g_rain;
        v[1] += g_scale;
    }
}

// Loss sensitivity at observation times: the state after step j is observed
// at sample s when sample_step[s][m] == j + 1; dL/dh += 2 (y - d) at the
// gauge cells.
__global__ void seed_kernel(const AdjArgs a, const int32_t* __restrict__ sample_step,
                            const float* __restrict__ y, const double* __restrict__ d,
                            const int32_t* __restrict__ cells, int ns, int G)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.M * G) return;
    const int m = t / G, g = t % G;
    const int j = a.seg_end[m] - 1 - a.rev_i;
    if (j < a.seg_first) return;
    float* lh = a.lam + ((size_t)a.lam_in * a.M + m) * 3 * a.plane;
    const int cell = cells[g];
    const size_t o = (size_t)(cell / a.nx) * a.ld + cell % a.nx;
    for (int s = 0; s < ns; ++s)
        if (sample_step[(size_t)s * a.M + m] == j + 1)
            lh[o] += (float)(2.0 * ((double)y[((size_t)s * a.M + m) * G + g] - d[(size_t)s * G + g]));
}

// Sum of the per-member Manning gradients in member order (deterministic).
__global__ void reduce_members_kernel(const float* __restrict__ gm, int M, int ny, int nx, int ld,
                                      size_t plane, float* __restrict__ out)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)ny * nx) return;
    const size_t r = t / nx, c = t % nx;
    const size_t o = r * ld + c;
    float acc = 0.0f;
    for (int m = 0; m < M; ++m) acc += gm[(size_t)m * plane + o];
    out[t] = acc;
}

}  // namespace

void launch_adjoint(const AdjArgs& a, int members_per_cta, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        adjoint_kernel<4, 1><<<grid, block, 0, s>>>(a);
    } else {
        dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
        adjoint_kernel<1, 4><<<grid, block, 0, s>>>(a);
    }
}

void launch_seed(const AdjArgs& a, const int32_t* sample_step, const float* y, const double* d,
                 const int32_t* cells, int ns, int G, cudaStream_t s)
{
    const int n = a.M * G;
    seed_kernel<<<(n + 127) / 128, 128, 0, s>>>(a, sample_step, y, d, cells, ns, G);
}

void launch_reduce_members(const float* gm, int M, int ny, int nx, int ld, size_t plane, float* out,
                           cudaStream_t s)
{
    const size_t n = (size_t)ny * nx;
    reduce_members_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gm, M, ny, nx, ld, plane, out);
}

}  // namespace flood
