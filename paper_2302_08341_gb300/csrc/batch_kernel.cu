// Batched step over uneven scenarios: every warp takes one task (a span of a
// strip of one scenario's grid) from a flat task table, plans the step of
// its scenario from the scenario's own clock (Eq. 4 on its own maximum
// depth, so each scenario has its own step length), and runs the same fused
// march as the ensemble kernel.  Scenarios that reached min(window end, own
// end time) are idle.
#include "batch.cuh"
#include "march.cuh"
#include "tma_march.cuh"

namespace flood {

namespace {


// Per-scenario plan (one thread per scenario, FP64): its own Eq. 4 step
// toward min(window end, own end time), clock, rain volume.
__global__ void batch_plan_kernel(const BatchArgs a, int n_scen)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_scen) return;
    const ScenDesc sd = a.scen[i];
    const MemberClock in = a.ms_in[i];
    const double t_stop = *a.t_stop;
    const double t_end = sd.t_end < t_stop ? sd.t_end : t_stop;
    const StepPlan sp = plan_step_p(a.alpha_dx, a.g, a.dt_cap, a.dt_fixed, a.h_floor, a.rain_block,
                                    t_end, sd.hyeto, sd.nb, sd.rain_mult, in);
    MemberPlan p;
    fill_plan(p, sp, a.g, a.dxd);
    p.cur = in.cur;
    p.ckpt = -1;
    a.ms_clr[i].hmax_bits = 0u;
    if (!sp.active) {
        a.ms_out[i] = in;
    } else {
        a.ms_out[i].t = sp.t_next;
        a.ms_out[i].steps = in.steps + 1;
        a.ms_out[i].cur = 1 - in.cur;
        a.rain_acc[i] += (double)sp.dr * a.cell_area * sd.ncell;
    }
    a.plan[i] = p;
}

template <int W>
__global__ void __launch_bounds__(32 * W) batch_step_kernel(const BatchArgs a)
{
    const int lane = threadIdx.x;
    const int tid = blockIdx.x * W + threadIdx.y;
    if (tid >= a.ntasks) return;
    const WarpTask tk = a.tasks[tid];
    const int i = tk.scen;
    const MemberPlan p = a.plan[i];
    if (!p.active) return;
    const ScenDesc sd = a.scen[i];
    FaceK k;
    k.gdt_dx = p.gdt_dx;
    k.gdt = p.gdt;
    k.dx_4dt = p.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = 0.0f;  // no inflow boundary here
    k.in_r0 = k.in_r1 = 0;
    const size_t ms = 3 * sd.plane;
    const float* src = sd.state + (size_t)p.cur * ms;
    float* dst = sd.state + (size_t)(1 - p.cur) * ms;
    const MarchOut mo = march_rows(src, dst, nullptr, nullptr, sd.z, sd.n, sd.plane, sd.ny, sd.nx, sd.ld, tk.c0,
                                   tk.r0, tk.r1, lane, k, p.dt_dx, sd.scale, p.dr, a.east_out,
                                   a.south_out);
    if (mo.bad) atomicOr(a.err, 1);
    const unsigned hb = __reduce_max_sync(0xffffffffu, mo.bad ? 0u : __float_as_uint(mo.hmax) & 0x7fffffffu);
    double out_acc = (double)mo.out_s - (double)mo.out_c, clamp_acc = (double)mo.clamp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        out_acc += __shfl_xor_sync(0xffffffffu, out_acc, off);
        clamp_acc += __shfl_xor_sync(0xffffffffu, clamp_acc, off);
    }
    if (lane == 0) {
        atomicMax(&a.ms_out[i].hmax_bits, hb);
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            double* v = a.vacc + (size_t)tk.slot * 2;
            v[0] += out_acc * p.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
    }
}

// TMA-staged form of batch_step_kernel (same results, bit for bit): the
// task's rows stream through shared memory by the scenario's own tensor maps.
template <int W, int LIM>
__global__ void __launch_bounds__(32 * W, 20 / W) batch_tma_kernel(const BatchArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const int tid = blockIdx.x * W + w;
    if (tid >= a.ntasks) return;  // whole warps; no block-wide barriers below
    const WarpTask tk = a.tasks[tid];
    const int i = tk.scen;
    const MemberPlan p = a.plan[i];
    if (!p.active) return;
    if (*reinterpret_cast<volatile const int*>(a.err) & 2) return;  // an earlier wait gave up
    const ScenDesc sd = a.scen[i];
    FaceK k;
    k.gdt_dx = p.gdt_dx;
    k.gdt = p.gdt;
    k.dx_4dt = p.dx_4dt;
    k.h_eps = a.h_eps;
    k.edge_drop = a.edge_drop;
    k.limiter = a.limiter;
    k.q_in = 0.0f;  // no inflow boundary here
    k.in_r0 = k.in_r1 = 0;
    uint32_t bar0;
    unsigned char* my_stages;
    tma_march_smem(smem_raw, W, w, bar0, my_stages);
    float* dst = sd.state + (size_t)(1 - p.cur) * 3 * sd.plane;
    MarchOut mo;
    if (!tma_march<false, false, LIM>(a.maps + 2 * i, a.maps + 2 * i + 1, p.cur * 3, bar0, my_stages, dst, nullptr,
                   nullptr, a.err, sd.plane, sd.ny, sd.nx, sd.ld, tk.c0, tk.r0, tk.r1, lane, k, p.dt_dx,
                   sd.scale, p.dr, a.east_out, a.south_out, mo))
        return;
    if (mo.bad) atomicOr(a.err, 1);
    const unsigned hb = __reduce_max_sync(0xffffffffu, mo.bad ? 0u : __float_as_uint(mo.hmax) & 0x7fffffffu);
    double out_acc = (double)mo.out_s - (double)mo.out_c, clamp_acc = (double)mo.clamp;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        out_acc += __shfl_xor_sync(0xffffffffu, out_acc, off);
        clamp_acc += __shfl_xor_sync(0xffffffffu, clamp_acc, off);
    }
    if (lane == 0) {
        atomicMax(&a.ms_out[i].hmax_bits, hb);
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            double* v = a.vacc + (size_t)tk.slot * 2;
            v[0] += out_acc * p.dt * a.dxd;
            v[1] += clamp_acc * a.cell_area;
        }
    }
}

}  // namespace

int batch_tma_prepare()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {batch_tma_kernel<4, 0>, batch_tma_kernel<4, 1>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma_march_smem_bytes(4));
    for (auto f : {batch_tma_kernel<8, 0>, batch_tma_kernel<8, 1>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma_march_smem_bytes(8));
    return e == cudaSuccess ? 0 : -1;
}

// the limiter is fixed at compile time (one instantiation per setting)
void launch_batch_step_tma(const BatchArgs& a, int warps_per_cta, cudaStream_t s)
{
    const unsigned g8 = (a.ntasks + 7) / 8, g4 = (a.ntasks + 3) / 4;
    if (warps_per_cta >= 8) {
        if (a.limiter)
            batch_tma_kernel<8, 1><<<g8, dim3(32, 8), tma_march_smem_bytes(8), s>>>(a);
        else
            batch_tma_kernel<8, 0><<<g8, dim3(32, 8), tma_march_smem_bytes(8), s>>>(a);
    } else {
        if (a.limiter)
            batch_tma_kernel<4, 1><<<g4, dim3(32, 4), tma_march_smem_bytes(4), s>>>(a);
        else
            batch_tma_kernel<4, 0><<<g4, dim3(32, 4), tma_march_smem_bytes(4), s>>>(a);
    }
}

void launch_batch_plan(const BatchArgs& a, int n_scen, cudaStream_t s)
{
    batch_plan_kernel<<<(n_scen + 127) / 128, 128, 0, s>>>(a, n_scen);
}

void launch_batch_step(const BatchArgs& a, int warps_per_cta, cudaStream_t s)
{
    if (warps_per_cta >= 8) {
        batch_step_kernel<8><<<(a.ntasks + 7) / 8, dim3(32, 8), 0, s>>>(a);
    } else {
        batch_step_kernel<4><<<(a.ntasks + 3) / 4, dim3(32, 4), 0, s>>>(a);
    }
}

}  // namespace flood
