// Fused local-inertial step: link fluxes (Eq. 2-3) and continuity (Eq. 5,
// Eq. 1) with rain, wet/dry clamp, the per-member maximum depth for the next
// Eq. 4 step, and the FP64 outflow / clamp volume partials, in one pass over
// the state.
//
// Work decomposition.  One warp owns a 128-column span (32 lanes x 4 cells,
// float4 loads and stores) of a strip of rows of ONE member and marches down
// the strip row by row.  A lane keeps the current row's depth, bed and
// roughness in registers, loads the next row (for the south links), computes
// the east and south links of its four cells, takes the west link from the
// neighbouring lane by shuffle and the north link from the previous row, and
// writes the new depth and both links.  Halo links (the north link of the
// strip's first row, the west link of the span's first column) are recomputed
// from the old state with the same rounded arithmetic as their owner, so both
// sides agree bit for bit.  A CTA holds WM members x WC spans; the WM warps of
// one span read the same bed and roughness lines, so those come from L1 once
// per tile for several members (Section 3.2's sharing of definitive data).
//
// HBM traffic per member-cell-step: read h, qx, qy (12 B), write h, qx, qy
// (12 B); z and n (8 B) once per tile for the WM members.
#include "flood_internal.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;  // columns per warp

__device__ __forceinline__ void load4(float (&v)[4], const float* p)
{
    float4 t = ldg4(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void store4(float* p, const float (&v)[4])
{
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

#ifndef FLOOD_STEP_MIN_BLOCKS
#define FLOOD_STEP_MIN_BLOCKS 6
#endif

// REPLAY = false: an ordinary step (per-member clock, Eq. 4 step length,
// reductions, optional logging and checkpoints).  REPLAY = true: recompute
// a recorded step of a checkpointed segment, bit for bit, for the adjoint.
template <int WM, int WC, bool REPLAY>
__global__ void __launch_bounds__(32 * WM * WC, FLOOD_STEP_MIN_BLOCKS * 4 / (WM * WC)) step_kernel(const StepArgs a)
{
    const int lane = threadIdx.x;
    const int wm = threadIdx.y % WM;
    const int wc = threadIdx.y / WM;
    const int m = blockIdx.x * WM + wm;
    const int span = blockIdx.y * WC + wc;
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps only: no block barriers below

    const int nx = a.nx, ny = a.ny, ld = a.ld;
    const size_t plane = a.plane;
    const size_t mstride = 3 * plane;
    const bool designated = (blockIdx.y == 0 && blockIdx.z == 0 && wc == 0 && lane == 0);
    StepPlan sp;
    const float* src;
    float* dst;
    float* ck = nullptr;
    if (REPLAY) {
        const int j = a.seg_first + a.replay_i;
        if (j >= a.seg_end[m]) return;
        sp.dt = a.dt_log[(size_t)m * a.dt_log_cap + j];
        sp.rdt = a.rdt_log[(size_t)m * a.dt_log_cap + j];
        sp.dr = (float)__dmul_rn(sp.rdt, (double)a.rain_mult[m]);
        dst = a.seg + ((size_t)(a.replay_i + 1) * a.M + m) * mstride;
        src = dst - (size_t)a.M * mstride;
    } else {
        const MemberClock in = a.ms_in[m];
        sp = plan_step(a, in, m);
        if (!sp.active) {
            if (designated) {
                a.ms_out[m] = in;
                a.ms_clr[m].hmax_bits = 0u;
            }
            return;
        }
        if (designated) {
            a.ms_out[m].t = sp.t_next;
            a.ms_out[m].steps = in.steps + 1;
            a.ms_out[m].cur = 1 - in.cur;  // hmax_bits: filled by atomicMax (slot was cleared)
            a.ms_clr[m].hmax_bits = 0u;
            a.rain_acc[m] += (double)sp.dr * a.cell_area * a.ncell;
            if (a.dt_log && in.steps < a.dt_log_cap) {
                a.dt_log[(size_t)m * a.dt_log_cap + in.steps] = sp.dt;
                a.rdt_log[(size_t)m * a.dt_log_cap + in.steps] = sp.rdt;
            }
        }
        src = a.state + (size_t)(in.cur * a.M + m) * mstride;
        dst = a.state + (size_t)((1 - in.cur) * a.M + m) * mstride;
        if (a.ckpt && (in.steps + 1) % a.ckpt_every == 0 && in.steps + 1 <= a.dt_log_cap)
            ck = a.ckpt + ((size_t)((in.steps + 1) / a.ckpt_every) * a.M + m) * mstride;
    }

    FaceK k;
    k.gdt_dx = (float)(a.g * sp.dt / a.dxd);
    k.gdt = (float)(a.g * sp.dt);
    k.dx_4dt = (float)(a.dxd / (4.0 * sp.dt));
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    const float dt_dx = (float)(sp.dt / a.dxd);
    const float s = a.scale[m];
    const float s_half = 0.5f * s;
    const float dr = sp.dr;

    const float* __restrict__ sh = src;
    const float* __restrict__ sqx = src + plane;
    const float* __restrict__ sqy = src + 2 * plane;
    float* __restrict__ dh = dst;
    float* __restrict__ dqx = dst + plane;
    float* __restrict__ dqy = dst + 2 * plane;
    const float* __restrict__ z = a.z;
    const float* __restrict__ n = a.n;

    const int c = c0 + 4 * lane;
    const bool act = c < nx;           // lane owns at least one real cell
    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, ny);
    const bool east_halo = (lane == 31) && (c + 4 < nx);

    float hC[4] = {0, 0, 0, 0}, zC[4] = {0, 0, 0, 0}, nC[4] = {0, 0, 0, 0};
    float qyN[4] = {0, 0, 0, 0};
    if (act) {
        const size_t o = (size_t)r0 * ld + c;
        load4(hC, sh + o);
        load4(zC, z + o);
        load4(nC, n + o);
        if (r0 > 0) {
            float hU[4], zU[4], nU[4], qU[4];
            const size_t ou = o - ld;
            load4(hU, sh + ou);
            load4(zU, z + ou);
            load4(nU, n + ou);
            load4(qU, sqy + ou);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                qyN[j] = (c + j < nx)
                             ? link_q(hU[j], zU[j], hC[j], zC[j], qU[j],
                                      __fmul_rn(s_half, __fadd_rn(nU[j], nC[j])), k)
                             : 0.0f;
        }
    }

    float hmax = 0.0f;
    bool bad = false;
    double out_acc = 0.0, clamp_acc = 0.0;

    for (int r = r0; r < r1; ++r) {
        const size_t o = (size_t)r * ld + c;
        const bool has_s = (r + 1 < ny);
        float hS[4] = {0, 0, 0, 0}, zS[4] = {0, 0, 0, 0}, nS[4] = {0, 0, 0, 0};
        float qxo[4] = {0, 0, 0, 0}, qyo[4] = {0, 0, 0, 0};
        if (act) {
            if (has_s) {
                load4(hS, sh + o + ld);
                load4(zS, z + o + ld);
                load4(nS, n + o + ld);
            }
            load4(qxo, sqx + o);
            load4(qyo, sqy + o);
        }
        // east neighbour of the lane's last cell: next lane's first cell
        float hE = __shfl_down_sync(0xffffffffu, hC[0], 1);
        float zE = __shfl_down_sync(0xffffffffu, zC[0], 1);
        float nE = __shfl_down_sync(0xffffffffu, nC[0], 1);
        if (east_halo) {
            const size_t oe = (size_t)r * ld + c + 4;
            hE = __ldg(sh + oe);
            zE = __ldg(z + oe);
            nE = __ldg(n + oe);
        }
        // east links (Eq. 2-3)
        float qxE[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cj = c + j;
            const float h2 = (j < 3) ? hC[j + 1] : hE;
            const float z2 = (j < 3) ? zC[j + 1] : zE;
            const float n2 = (j < 3) ? nC[j + 1] : nE;
            float q;
            if (cj < nx - 1)
                q = link_q(hC[j], zC[j], h2, z2, qxo[j], __fmul_rn(s_half, __fadd_rn(nC[j], n2)), k);
            else if (cj == nx - 1)
                q = a.east_out ? outflow_q(hC[j], qxo[j], __fmul_rn(s, nC[j]), k) : 0.0f;
            else
                q = 0.0f;
            qxE[j] = q;
        }
        // west link of the lane's first cell: previous lane's last east link
        float qW0 = __shfl_up_sync(0xffffffffu, qxE[3], 1);
        if (lane == 0) {
            qW0 = 0.0f;
            if (c0 > 0) {  // recompute the neighbouring span's link (halo)
                const size_t ow = (size_t)r * ld + c0 - 1;
                qW0 = link_q(__ldg(sh + ow), __ldg(z + ow), hC[0], zC[0], __ldg(sqx + ow),
                             __fmul_rn(s_half, __fadd_rn(__ldg(n + ow), nC[0])), k);
            }
        }
        // south links (Eq. 2-3)
        float qyS[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cj = c + j;
            float q = 0.0f;
            if (cj < nx) {
                if (has_s)
                    q = link_q(hC[j], zC[j], hS[j], zS[j], qyo[j],
                               __fmul_rn(s_half, __fadd_rn(nC[j], nS[j])), k);
                else if (a.south_out)
                    q = outflow_q(hC[j], qyo[j], __fmul_rn(s, nC[j]), k);
            }
            qyS[j] = q;
        }
        // continuity (Eq. 5 -> Eq. 1) with rain and the wet/dry clamp
        float hN[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cj = c + j;
            float hn = 0.0f;
            if (cj < nx) {
                const float qW = (j == 0) ? qW0 : qxE[j - 1];
                const float net = __fadd_rn(__fsub_rn(qW, qxE[j]), __fsub_rn(qyN[j], qyS[j]));
                hn = __fadd_rn(__fmaf_rn(dt_dx, net, hC[j]), dr);
                if (hn < 0.0f) {
                    // clamped cells keep a negative zero: the adjoint reads
                    // the sign bit to know this branch was taken
                    clamp_acc -= (double)hn;
                    hn = -0.0f;
                }
                bad |= !(hn <= 3.0e38f);  // NaN or overflow
                hmax = fmaxf(hmax, hn);
                if (cj == nx - 1 && a.east_out) out_acc += (double)qxE[j];
                if (!has_s && a.south_out) out_acc += (double)qyS[j];
            }
            hN[j] = hn;
        }
        if (act) {
            store4(dh + o, hN);
            store4(dqx + o, qxE);
            store4(dqy + o, qyS);
            if (ck) {
                store4(ck + o, hN);
                store4(ck + plane + o, qxE);
                store4(ck + 2 * plane + o, qyS);
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
    }

    // warp reductions: max depth (order-free), FP64 volumes in a fixed order
    if (bad) atomicOr(a.err, 1);
    if (REPLAY) return;
    const unsigned hb = __reduce_max_sync(0xffffffffu, __float_as_uint(hmax) & 0x7fffffffu);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        out_acc += __shfl_xor_sync(0xffffffffu, out_acc, off);
        clamp_acc += __shfl_xor_sync(0xffffffffu, clamp_acc, off);
    }
    if (lane == 0) {
        atomicMax(&a.ms_out[m].hmax_bits, hb);
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            const int slot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
            double* v = a.vacc + ((size_t)m * a.nslot + slot) * 2;
            v[0] += out_acc * sp.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
    }
}

}  // namespace

int step_nslot(int ny, int nx, int rows_per_strip)
{
    return ((ny + rows_per_strip - 1) / rows_per_strip) * ((nx + kSpan - 1) / kSpan);
}

// members_per_cta: warps of one CTA hold this many members of the same span
// (1: one member over 4 spans, for single members; 2: 2 members x 2 spans;
// 4 or 8: 4 or 8 members of one span).
void launch_step(const StepArgs& a, int members_per_cta, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    switch (members_per_cta) {
    case 8: {
        dim3 grid((a.M + 7) / 8, spans, strips), block(32, 8);
        step_kernel<8, 1, false><<<grid, block, 0, s>>>(a);
        break;
    }
    case 4: {
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        step_kernel<4, 1, false><<<grid, block, 0, s>>>(a);
        break;
    }
    case 2: {
        dim3 grid((a.M + 1) / 2, (spans + 1) / 2, strips), block(32, 4);
        step_kernel<2, 2, false><<<grid, block, 0, s>>>(a);
        break;
    }
    default: {
        dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
        step_kernel<1, 4, false><<<grid, block, 0, s>>>(a);
        break;
    }
    }
}

void launch_replay(const StepArgs& a, int members_per_cta, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        step_kernel<4, 1, true><<<grid, block, 0, s>>>(a);
    } else {
        dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
        step_kernel<1, 4, true><<<grid, block, 0, s>>>(a);
    }
}

}  // namespace flood
