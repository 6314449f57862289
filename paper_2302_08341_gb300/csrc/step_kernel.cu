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
#include "march.cuh"

namespace flood {

namespace {

constexpr int kSpan = 128;  // columns per warp

#ifndef FLOOD_STEP_MIN_BLOCKS
#define FLOOD_STEP_MIN_BLOCKS 6
#endif

// Per-member step plan (one thread per member, FP64): Eq. 4 step length,
// rain of the block, the member's clock in the next slot, the rain volume and
// (when logging) the step record and checkpoint slot.
__global__ void plan_kernel(const StepArgs a)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.M) return;
    const MemberClock in = a.ms_in[m];
    const StepPlan sp = plan_step(a, in, m);
    MemberPlan p;
    fill_plan(p, sp, a.g, a.dxd);
    p.cur = in.cur;
    p.ckpt = -1;
    p.q_in = 0.0f;
    if (a.inflow && sp.active) {  // the block's discharge spread over the inflow rows
        const double blk = floor(__ddiv_rn(in.t, a.rain_block));
        const int b = (int)blk;
        const double Q = (blk >= 0.0 && b < a.inflow_blocks) ? (double)a.inflow[b] : 0.0;
        p.q_in = (float)(Q / (a.dxd * (double)(a.in_r1 - a.in_r0)));
        a.inflow_acc[m] += (double)p.q_in * a.dxd * (double)(a.in_r1 - a.in_r0) * sp.dt;
    }
    a.ms_clr[m].hmax_bits = 0u;  // the slot the next step's maximum goes to
    if (!sp.active) {
        a.ms_out[m] = in;
        a.plan[m] = p;
        return;
    }
    a.ms_out[m].t = sp.t_next;
    a.ms_out[m].steps = in.steps + 1;
    a.ms_out[m].cur = 1 - in.cur;  // hmax_bits: atomicMax by the step kernel (slot was cleared)
    a.rain_acc[m] += (double)sp.dr * a.cell_area * a.ncell;
    if (a.ckpt && (in.steps + 1) % a.ckpt_every == 0 && in.steps + 1 <= a.dt_log_cap)
        p.ckpt = (int)((in.steps + 1) / a.ckpt_every);
    if (a.log && in.steps < a.dt_log_cap) a.log[(size_t)m * a.dt_log_cap + in.steps] = p;
    a.plan[m] = p;
}

// REPLAY = false: an ordinary step with the plan of this step.  REPLAY =
// true: recompute a logged step of a checkpointed segment, bit for bit, for
// the adjoint.
template <int WM, int WC, bool REPLAY, bool LC = false>
__global__ void __launch_bounds__(32 * WM * WC, (LC ? 4 : FLOOD_STEP_MIN_BLOCKS) * 4 / (WM * WC))
    step_kernel(const StepArgs a)
{
    const int lane = threadIdx.x;
    const int wm = threadIdx.y % WM;
    const int wc = threadIdx.y / WM;
    const int m = a.m_base + blockIdx.x * WM + wm;
    const int span = blockIdx.y * WC + wc;
    const int c0 = span * kSpan;
    if (m >= a.M || c0 >= a.nx) return;  // whole warps only: no block barriers below

    const int nx = a.nx, ny = a.ny, ld = a.ld;
    const size_t plane = a.plane;
    const size_t mstride = 3 * plane;
    MemberPlan p;
    const float* src;
    float* dst;
    float* ck = nullptr;
    if (REPLAY) {
        const int j = a.seg_first + a.replay_i;
        if (j >= a.seg_end[m]) return;
        p = a.log[(size_t)m * a.dt_log_cap + j];
        dst = a.seg + ((size_t)(a.replay_i + 1) * a.M + m) * mstride;
        src = dst - (size_t)a.M * mstride;
    } else {
        p = a.plan[m];
        if (!p.active) return;
        src = a.state + (size_t)(p.cur * a.M + m) * mstride;
        dst = a.state + (size_t)((1 - p.cur) * a.M + m) * mstride;
        if (p.ckpt >= 0) ck = a.ckpt + ((size_t)p.ckpt * a.M + m) * mstride;
    }
    FaceK k;
    k.gdt_dx = p.gdt_dx;
    k.gdt = p.gdt;
    k.dx_4dt = p.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = p.q_in;
    k.in_r0 = a.in_r0;
    k.in_r1 = a.in_r1;

    const int r0 = blockIdx.z * a.rows_per_strip;
    const int r1 = min(r0 + a.rows_per_strip, ny);
    float* hm = (!REPLAY && a.hmax_field) ? a.hmax_field + (size_t)m * plane : nullptr;
    LandK lk;
    if (LC) lk = land_k(a, m, p.dr, p.dt, lane);
    const MarchOut mo = march_rows<LC>(src, dst, ck, hm, a.z, a.n, plane, ny, nx, ld, c0, r0, r1,
                                       lane, k, p.dt_dx, a.scale[m], p.dr, a.east_out, a.south_out,
                                       &lk);
    if (mo.bad) atomicOr(a.err, 1);
    if (REPLAY) return;
    // warp reductions: max depth (order-free); volume partials widened to
    // FP64 once per warp and reduced in a fixed order
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
        const int slot = blockIdx.z * ((a.nx + kSpan - 1) / kSpan) + span;
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            double* v = a.vacc + ((size_t)m * a.nslot + slot) * 2;
            v[0] += out_acc * p.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
        if (LC && drn_acc != 0.0) a.dacc[(size_t)m * a.nslot + slot] += drn_acc * a.cell_area;
    }
}

}  // namespace

void launch_plan(const StepArgs& a, cudaStream_t s)
{
    plan_kernel<<<(a.M + 127) / 128, 128, 0, s>>>(a);
}

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
    if (a.lc_on) {  // land cover: 4 members per CTA, or one member over 4 spans
        if (members_per_cta >= 4) {
            dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
            step_kernel<4, 1, false, true><<<grid, block, 0, s>>>(a);
        } else {
            dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
            step_kernel<1, 4, false, true><<<grid, block, 0, s>>>(a);
        }
        return;
    }
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

// The plain form, for comparison: one launch per member per step, each
// covering one member's grid with 4 spans per CTA (as a single deterministic
// model would be launched), so the bed and roughness are read once per member.
void launch_step_per_member(const StepArgs& a, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    dim3 grid(1, (spans + 3) / 4, strips), block(32, 4);
    StepArgs b = a;
    for (int m = 0; m < a.M; ++m) {
        b.m_base = m;
        step_kernel<1, 4, false><<<grid, block, 0, s>>>(b);
    }
}

void launch_replay(const StepArgs& a, int members_per_cta, cudaStream_t s)
{
    const int spans = (a.nx + kSpan - 1) / kSpan;
    const int strips = (a.ny + a.rows_per_strip - 1) / a.rows_per_strip;
    if (members_per_cta >= 4) {
        dim3 grid((a.M + 3) / 4, spans, strips), block(32, 4);
        if (a.lc_on)
            step_kernel<4, 1, true, true><<<grid, block, 0, s>>>(a);
        else
            step_kernel<4, 1, true><<<grid, block, 0, s>>>(a);
    } else {
        dim3 grid(a.M, (spans + 3) / 4, strips), block(32, 4);
        if (a.lc_on)
            step_kernel<1, 4, true, true><<<grid, block, 0, s>>>(a);
        else
            step_kernel<1, 4, true><<<grid, block, 0, s>>>(a);
    }
}

}  // namespace flood
