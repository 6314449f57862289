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
#include "adjoint_row.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;

__device__ __forceinline__ void load4(float (&v)[4], const float* p)
{
    float4 t = ldg4(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// RW: land cover (per-member Manning n fields, rain weighed by the runoff
// coefficient, drainage partials), with the registers of three CTAs per SM.
template <int WM, int WC, int LIM, bool RW = false>
__global__ void __launch_bounds__(32 * WM * WC, RW ? 3 : 4) adjoint_kernel(const AdjArgs a)
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
    k.q_in = 0.0f;  // no inflow boundary here
    k.in_r0 = k.in_r1 = 0;
    const float T = pl.dt_dx;
    const float s = a.scale[m];
    const float s_half = 0.5f * s;
    const bool interior = c0 + kSpan < nx;  // no east edge in this span

    const float* __restrict__ st = a.seg + ((size_t)(j - a.seg_first) * a.M + m) * mstride;
    const float* __restrict__ sh = st;
    const float* __restrict__ sqx = st + plane;
    const float* __restrict__ sqy = st + 2 * plane;
    const float* __restrict__ h1p = st + (size_t)a.M * mstride;  // depth after the step
    const float* __restrict__ z = a.z;
    const float* __restrict__ n = a.n + (size_t)m * a.n_mstride;
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
            float hU[4], zU[4], nU[4], qU[4], lqU[4], haU[4], lhU[4], lU[4];
            load4(hU, sh + u); load4(zU, z + u); load4(nU, n + u); load4(qU, sqy + u);
            load4(lqU, lin + 2 * plane + u); load4(haU, h1p + u); load4(lhU, lin + u);
#pragma unroll
            for (int q = 0; q < 4; ++q) lU[q] = masked(haU[q], lhU[q]);
            north_carry<LIM>(hU, zU, nU, qU, lqU, lU, hC, zC, nC, lC, c, nx, s_half, T, k, carH,
                             carN);
        }
    }

    // FP32 compensated sums of the rows' partials (lambda~ for the rain
    // gradient, mu n dq'/dn for the scale gradient), widened to FP64 once per warp
    float gr_s = 0.0f, gr_c = 0.0f, gs_s = 0.0f, gs_c = 0.0f;
    float gd_s = 0.0f, gd_c = 0.0f;  // land cover: drainage partials
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
        WestIn wi{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (lane == 0 && c0 > 0) {
            const size_t w = o - 1;
            wi.h = __ldg(sh + w); wi.z = __ldg(z + w); wi.n = __ldg(n + w);
            wi.qx = __ldg(sqx + w); wi.lqx = __ldg(lin + plane + w);
            wi.l = masked(__ldg(h1p + w), __ldg(lin + w));
        }
        float lh[4], lx[4], ly[4], gnr[4];
        float gr_row = 0.0f, gs_row = 0.0f;
        float rwv[4] = {0, 0, 0, 0};
        if (RW) {
            float dfv[4] = {0, 0, 0, 0}, haC[4] = {0, 0, 0, 0};
            if (act) {
                load4(rwv, a.rw + o);
                load4(dfv, a.dflag + o);
                load4(haC, h1p + o);
            }
            kahan_add(gd_s, gd_c, drain_row(lC, haC, dfv));
        }
        if (interior)
            adjoint_row<true, LIM, RW>(hC, zC, nC, lC, hS, zS, nS, lS, qxo, qyo, lqx, lqy, hE, zE,
                                       nE, lE, c0 > 0, wi, has_s, c, nx, lane, s, s_half, T, k,
                                       a.east_out, a.south_out, carH, carN, gr_row, gs_row, lh, lx,
                                       ly, gnr, rwv);
        else
            adjoint_row<false, LIM, RW>(hC, zC, nC, lC, hS, zS, nS, lS, qxo, qyo, lqx, lqy, hE, zE,
                                        nE, lE, c0 > 0, wi, has_s, c, nx, lane, s, s_half, T, k,
                                        a.east_out, a.south_out, carH, carN, gr_row, gs_row, lh, lx,
                                        ly, gnr, rwv);
        kahan_add(gr_s, gr_c, gr_row);
        kahan_add(gs_s, gs_c, gs_row);
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
    const int slot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
    adjoint_partials(a.gpart, a.nslot, m, slot, lane, gr_s, gr_c, gs_s, gs_c, pl.rdt,
                     1.0 / (double)s);
    if (RW) adjoint_drain_partial(a.gdpart, a.nslot, m, slot, lane, gd_s, gd_c, pl.dt);
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

template <int LIM, bool RW>
void launch_adjoint_lim(const AdjArgs& a, int members_per_cta, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        adjoint_kernel<4, 1, LIM, RW><<<grid, block, 0, s>>>(a);
    } else {
        dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
        adjoint_kernel<1, 4, LIM, RW><<<grid, block, 0, s>>>(a);
    }
}

}  // namespace

void launch_adjoint(const AdjArgs& a, int members_per_cta, cudaStream_t s)
{
    if (a.rw)
        a.limiter ? launch_adjoint_lim<1, true>(a, members_per_cta, s)
                  : launch_adjoint_lim<0, true>(a, members_per_cta, s);
    else
        a.limiter ? launch_adjoint_lim<1, false>(a, members_per_cta, s)
                  : launch_adjoint_lim<0, false>(a, members_per_cta, s);
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
