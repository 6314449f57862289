// Internal definitions shared by the CUDA translation units of libflood.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/flood.h"

namespace flood {

// Default limit of a bounded mbarrier wait for a staged tile, in SM clock
// cycles (about 0.1 s).
constexpr long long kTmaWaitBudgetDefault = 200000000LL;

// Per-member scalars.  Kept in three rotating slots so that a step kernel can
// read its inputs from one slot, build the next slot (the new clock, the new
// maximum depth by atomicMax) and clear the slot after that, without any
// grid-wide synchronisation: step k reads slot k%3, writes slot (k+1)%3 and
// clears the maximum of slot (k+2)%3.
struct MemberClock {
    double t;           // simulated time (s)
    int64_t steps;      // steps taken by this member
    uint32_t hmax_bits; // max depth of the current state (non-negative float bits)
    int32_t cur;        // which of the two state buffers holds the current state
};

// Everything a step launch needs, passed by value.
struct StepArgs {
    float* state;               // [2][M][3][plane]: h, qx, qy planes, two buffers
    const float* z;             // [ny][ld]
    const float* n;             // [ny][ld]
    const float* rain_mult;     // [M]
    const float* scale;         // [M]
    const float* hyeto;         // [nb] rain rate per block (m/s)
    const MemberClock* ms_in;   // slot k%3
    MemberClock* ms_out;        // slot (k+1)%3
    MemberClock* ms_clr;        // slot (k+2)%3
    double* vacc;               // [M][nslot][2] outflow and clamp partial volumes
    double* rain_acc;           // [M] rain volume added
    struct MemberPlan* plan;    // [M] this step's plan of every member (plan kernel -> step kernel)
    struct MemberPlan* log;     // [M][dt_log_cap] plans of the steps taken (or null)
    float* ckpt;                // [n_ckpt][M][3][plane] checkpoint states (or null)
    int ckpt_every;             // a checkpoint after every ckpt_every steps of a member
    // replay of a checkpointed segment (adjoint recomputation): slot i of
    // seg holds the state after step seg_first + i; this launch recomputes
    // step seg_first + replay_i of every member with seg_first + replay_i <
    // seg_end[m], with the recorded step length and rain
    float* seg;                 // [slots][M][3][plane]
    const int* seg_end;         // [M]
    int seg_first, replay_i;
    int* err;                   // device error word (bit 0: non-finite depth)
    long long wait_budget;      // clock cycles a TMA row wait of the step may take
    int m_base;                 // first member of this launch (one-launch-per-member form)
    float* hmax_field;          // [M][plane] running maximum depth (or null: not tracked)
    // land cover (Section 4.1; lc_on = 0: none)
    int lc_on;
    const uint8_t* cls;         // [ny][ld] class of every cell (< 4)
    const float* lc_n;          // [M][4] Manning n of each class, per member
    const float* lc_drain;      // [M] drainage rate (m/s), per member
    float lc_runoff[4];         // fraction of the rain that stays, per class
    float lc_drains[4];         // 1: the member's drainage applies to the class
    double* dacc;               // [M][nslot] drained volume partials
    // inflow hydrograph through west-edge rows [in_r0, in_r1) (inflow = null: none)
    const float* inflow;        // [inflow_blocks] discharge per rain block (m^3/s)
    int inflow_blocks, in_r0, in_r1;
    double* inflow_acc;         // [M] inflow volume
    // tiles of the ordinary TMA step (null: every (span, strip) tile): the
    // (span, strip) of each tile holding a cell of the domain; the others
    // lie wholly outside it, where the state stays zero
    const int2* tiles;
    int n_tiles;
    size_t plane;               // ny * ld
    int ny, nx, ld, M, nb;
    int rows_per_strip;
    int nslot;                  // slots per member in vacc
    int dt_log_cap;
    double t_end;               // < 0: no end
    double alpha_dx;            // k * dx of Eq. 4
    double g;
    double dt_cap, dt_fixed, h_floor, rain_block;
    double dxd;                 // dx (FP64)
    double cell_area;           // dx * dx
    double ncell;               // ny * nx
    float dx, h_eps, edge_drop; // edge_drop = edge_slope * dx
    int limiter, east_out, south_out;
};

// Arguments of the TMA-staged step kernel: tensor maps of the two state
// buffers ([2 M 3] planes of [ny][ld]) and of the static fields ([z, n]
// planes; with land cover [z, class code]), 3-D tiles of 136 columns x 1 row
// x (3 or 2) planes.
struct TmaArgs {
    CUtensorMap state_map;
    CUtensorMap static_map;
    CUtensorMap hm_map;     // running maxima (ld, ny, M), box 128 x 1 x 1 (tracking only)
    StepArgs a;
};

// One member's step, planned once per step in FP64 by the plan kernel and
// handed to the step kernels as FP32 constants (the step kernels themselves
// run no FP64 arithmetic: GB300's FP64 pipe is narrow).
struct MemberPlan {
    double t_next, dt, rdt;   // time after the step, step length, dt x block rain rate
    float dr;                 // rain depth added to every cell (m)
    float gdt_dx, gdt, dx_4dt, dt_dx;
    int active;               // 0: the member does not step
    int cur;                  // buffer holding the member's state before the step
    int ckpt;                 // checkpoint slot that also receives the result, or -1
    float q_in;               // inflow flux per unit width of this step (m^2/s), 0 without
};

// Step length of one member (Eq. 4 with floor, cap and landing on the next
// stop).  Every CTA of a member evaluates this identically in FP64.
struct StepPlan {
    double dt, t_next;
    double rdt;        // dt x rain rate of the block (m), before the member's multiplier
    float dr;          // rain depth added to every cell this step (m)
    bool active;
};

// Step plan from explicit scheme constants (shared by the ensemble and the
// batched kernels).
__device__ __forceinline__ StepPlan plan_step_p(double alpha_dx, double g, double dt_cap,
                                                double dt_fixed, double h_floor, double rain_block,
                                                double t_end, const float* hyeto, int nb,
                                                float rain_mult, const MemberClock& in)
{
    StepPlan s;
    s.active = !(t_end >= 0.0 && in.t >= t_end);
    double dt;
    if (dt_fixed > 0.0) {
        dt = dt_fixed;
    } else {
        double hm = (double)__uint_as_float(in.hmax_bits);
        hm = hm > h_floor ? hm : h_floor;
        dt = __ddiv_rn(alpha_dx, __dsqrt_rn(__dmul_rn(g, hm)));
        dt = dt > dt_cap ? dt_cap : dt;
    }
    double blk = floor(__ddiv_rn(in.t, rain_block));
    double stop = __dmul_rn(blk + 1.0, rain_block);
    if (t_end >= 0.0 && t_end < stop) stop = t_end;
    if (__dadd_rn(in.t, dt) >= stop) {
        dt = __dsub_rn(stop, in.t);
        s.t_next = stop;
    } else {
        s.t_next = __dadd_rn(in.t, dt);
    }
    s.dt = dt;
    int b = (int)blk;
    double rate = (blk >= 0.0 && b < nb) ? (double)hyeto[b] : 0.0;
    s.rdt = __dmul_rn(dt, rate);
    s.dr = (float)__dmul_rn(s.rdt, (double)rain_mult);
    return s;
}

__device__ __forceinline__ StepPlan plan_step(const StepArgs& a, const MemberClock& in, int m)
{
    return plan_step_p(a.alpha_dx, a.g, a.dt_cap, a.dt_fixed, a.h_floor, a.rain_block, a.t_end,
                       a.hyeto, a.nb, a.rain_mult[m], in);
}

__device__ __forceinline__ void fill_plan(MemberPlan& p, const StepPlan& sp, double g, double dxd)
{
    p.t_next = sp.t_next;
    p.dt = sp.dt;
    p.rdt = sp.rdt;
    p.dr = sp.dr;
    p.gdt_dx = (float)(g * sp.dt / dxd);
    p.gdt = (float)(g * sp.dt);
    p.dx_4dt = (float)(dxd / (4.0 * sp.dt));
    p.dt_dx = (float)(sp.dt / dxd);
    p.active = sp.active ? 1 : 0;
}

// Compensated (Kahan) FP32 summation for the per-warp volume partials; the
// explicit rounding intrinsics keep the compiler from re-associating it.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// Per-step constants of one member (FP32).
struct FaceK {
    float gdt_dx;     // g dt / dx
    float gdt;        // g dt
    float dx_4dt;     // dx / (4 dt): limiter factor
    float h_eps;      // no flow unless the flow depth exceeds this (0: Eq. 2-3 as printed)
    float edge_drop;  // bed drop over one cell past a free-outflow edge
    int limiter;
    float q_in;       // inflow flux per unit width through west-edge rows [in_r0, in_r1)
    int in_r0, in_r1;
};

// Hardware approximate base-2 logarithm, base-2 exponential and reciprocal
// (one special-function-unit instruction each, denormals flushed to zero).
__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// max that propagates a NaN operand (fmaxf returns the other one)
__device__ __forceinline__ float fmax_nan(float a, float b)
{
    float y;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// h^(-7/3) = 2^(-7/3 log2 h), capped so that h -> 0 (or h <= 0, which only
// occurs on links that carry no flow) gives a finite, huge friction factor
// and q = 0 still gives exactly zero friction.
__device__ __forceinline__ float inv_h73(float h)
{
    return fminf(ex2_approx(__fmul_rn(-2.33333333f, lg2_approx(h))), 1.0e30f);
}

// Eq. 2 given the flow depth hf, dx * S_surf (dS), the old flux q and the
// link roughness: q' = (q - g hf dt S) / (1 + g n^2 |q| dt / hf^(7/3)).
__device__ __forceinline__ float eq2(float hf, float dS, float q, float n_link, const FaceK& k)
{
    const float num = __fmaf_rn(-__fmul_rn(k.gdt_dx, hf), dS, q);
    const float c = __fmul_rn(__fmul_rn(k.gdt, __fmul_rn(n_link, n_link)), fabsf(q));
    const float fr = __fmul_rn(c, inv_h73(hf));
    return __fmul_rn(num, rcp_approx(__fadd_rn(1.0f, fr)));
}

// Eq. 3 then Eq. 2 on one interior link (cell 1 on the low-index side, cell
// 2 on the high-index side; positive flow from 1 to 2), then the
// quarter-volume limiter.  No flow unless the flow depth exceeds h_eps (0 by
// default: Eq. 2-3 as printed).  Straight-line code of explicitly rounded
// intrinsics, so a link computed twice (by the tile that owns it and, as a
// halo, by its neighbour) gives bit-identical values and the update stays
// exactly conservative.
// LIM: 1 or 0 fixes the limiter on or off at compile time (the step kernels
// instantiate both), -1 reads it from k.
template <int LIM = -1>
__device__ __forceinline__ float link_q(float h1, float z1, float h2, float z2, float q,
                                        float n_link, const FaceK& k)
{
    // h_flow = max(eta1, eta2) - max(z1, z2) = max(h1 - max(dz, 0), h2 + min(dz, 0))
    // with dz = z2 - z1: the large bed elevation cancels exactly
    const float dz = __fsub_rn(z2, z1);
    const float hf = fmaxf(__fsub_rn(h1, fmaxf(dz, 0.0f)), __fadd_rn(h2, fminf(dz, 0.0f)));
    // dx * S_surf = (z2 - z1) + (h2 - h1)
    const float dS = __fadd_rn(dz, __fsub_rn(h2, h1));
    float qn = eq2(hf, dS, q, n_link, k);
    if (LIM == 1 || (LIM < 0 && k.limiter)) {
        // |q'| <= h_upstream dx / (4 dt): with h1, h2 >= 0 the two one-sided
        // clamps equal the clamp by the depth of the cell the flow leaves
        qn = fmaxf(fminf(qn, __fmul_rn(h1, k.dx_4dt)), -__fmul_rn(h2, k.dx_4dt));
    }
    return hf > k.h_eps ? qn : 0.0f;
}

// Free-outflow edge link: a ghost cell continuing the bed at the edge slope
// with the edge cell's depth, so h_flow = h and dx * S = -edge_slope * dx;
// only outward flow passes.
template <int LIM = -1>
__device__ __forceinline__ float outflow_q(float h, float q, float n_cell, const FaceK& k)
{
    float qn = eq2(h, -k.edge_drop, q, n_cell, k);
    if (LIM == 1 || (LIM < 0 && k.limiter)) qn = fminf(qn, __fmul_rn(h, k.dx_4dt));
    return h > k.h_eps ? fmaxf(qn, 0.0f) : 0.0f;
}

__device__ __forceinline__ float4 ldg4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }

// Land cover of one member for one step (Section 4.1): per class, the
// Manning n, the rain depth that stays on the surface and the drainage
// depth.  Classes are 0..3, four to a 32-bit word (one lane's four cells).
// The four-entry tables live in lanes 0..3 (lane q holds class q & 3's
// entries) and are read by shuffle, so every lane of the warp must take
// part in each lookup.
struct LandK {
    const uint8_t* cls;  // [ny][ld]
    float n, dr, dd;     // this lane's entries: class (lane & 3)
};

__device__ __forceinline__ float land_get(float v, uint32_t k)
{
    return __shfl_sync(0xffffffffu, v, (int)k);
}

__device__ __forceinline__ uint32_t cls_word(const uint8_t* cls, size_t o)
{
    return *reinterpret_cast<const uint32_t*>(cls + o);
}

// Source lane of cell j's class-table entry, for land_get: the shuffle reads
// only the five low bits of its source lane, and class codes (< 4) fill the
// two low bits of their byte, so the byte needs no masking.
__device__ __forceinline__ uint32_t cls_at(uint32_t w, int j) { return w >> (8 * j); }

__device__ __forceinline__ void land_n4(float (&nv)[4], uint32_t w, const LandK& lk)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) nv[j] = land_get(lk.n, cls_at(w, j));
}

// The rain and drainage depths of a lane's four cells (whole warp).
__device__ __forceinline__ void land_src4(float (&drv)[4], float (&ddv)[4], uint32_t w,
                                          const LandK& lk)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        drv[j] = land_get(lk.dr, cls_at(w, j));
        ddv[j] = land_get(lk.dd, cls_at(w, j));
    }
}

// This member's land-cover tables for a step: dr = its rain depth, dt the
// step length.
__device__ __forceinline__ LandK land_k(const StepArgs& a, int m, float dr, double dt, int lane)
{
    LandK lk;
    lk.cls = a.cls;
    const int q = lane & 3;
    lk.n = a.lc_n[(size_t)m * 4 + q];
    lk.dr = __fmul_rn(dr, a.lc_runoff[q]);
    lk.dd = __fmul_rn(__fmul_rn(a.lc_drain[m], a.lc_drains[q]), (float)dt);
    return lk;
}

// Host-side helpers (flood_capi.cu).
void launch_plan(const StepArgs& a, cudaStream_t s);
void launch_step(const StepArgs& a, int members_per_cta, cudaStream_t s);
void launch_step_per_member(const StepArgs& a, cudaStream_t s);
void launch_replay(const StepArgs& a, int members_per_cta, cudaStream_t s);
int launch_step_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s);
// t.state_map over the adjoint's segment slots (box: 3 planes)
void launch_replay_tma(const TmaArgs& t, int members_per_cta, cudaStream_t s);
int tma_box_cols();
int encode_map_3d_u8(CUtensorMap* map, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
                     uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t b0, uint32_t b1,
                     uint32_t b2);
int step_nslot(int ny, int nx, int rows_per_strip);

}  // namespace flood
