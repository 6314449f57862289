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

// A task's reductions: the scenario's maximum depth (atomicMax into its next
// clock), the non-finite flag, and the task's outflow, clamp and (land
// cover) drained volume partials in its own slot.  ATOMIC: the slot may be
// updated from another SM in the same launch (persistent form).
template <bool LC, bool ATOMIC>
__device__ __forceinline__ void finish_task(const BatchArgs& a, MemberClock* ms_out, const WarpTask& tk,
                                            const MemberPlan& p, const MarchOut& mo, int lane)
{
    if (mo.bad) atomicOr(a.err, 1);
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
        atomicMax(&ms_out[tk.scen].hmax_bits, hb);
        if (out_acc != 0.0 || clamp_acc != 0.0) {
            double* v = a.vacc + (size_t)tk.slot * 2;
            if (ATOMIC) {
                atomicAdd(v, out_acc * p.dt * a.dxd);
                atomicAdd(v + 1, clamp_acc * a.cell_area);
            } else {
                v[0] += out_acc * p.dt * a.dxd;
                v[1] += clamp_acc * a.cell_area;
            }
        }
        if (LC && drn_acc != 0.0) {
            if (ATOMIC)
                atomicAdd(a.dacc + tk.slot, drn_acc * a.cell_area);
            else
                a.dacc[tk.slot] += drn_acc * a.cell_area;
        }
    }
}

template <int W, bool LC>
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
    LandK lk;
    if (LC) lk = batch_land_k(a.scen + i, p.dr, p.dt, lane);
    const MarchOut mo = march_rows<LC>(src, dst, nullptr, nullptr, sd.z, sd.n, sd.plane, sd.ny, sd.nx,
                                       sd.ld, tk.c0, tk.r0, tk.r1, lane, k, p.dt_dx, sd.scale, p.dr,
                                       a.east_out, a.south_out, &lk);
    finish_task<LC, false>(a, a.ms_out, tk, p, mo, lane);
}

// TMA-staged form of batch_step_kernel (same results, bit for bit): the
// task's rows stream through shared memory by the scenario's own tensor maps.
template <int W, int LIM, bool LC>
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
    LandK lk;
    if (LC) lk = batch_land_k(a.scen + i, p.dr, p.dt, lane);
    MarchOut mo;
    if (!tma_march<false, LC, LIM>(a.maps + 2 * i, a.maps + 2 * i + 1, p.cur * 3, bar0, my_stages,
                                   dst, nullptr, nullptr, a.err, sd.plane, sd.ny, sd.nx, sd.ld, tk.c0,
                                   tk.r0, tk.r1, lane, k, p.dt_dx, sd.scale, p.dr, a.east_out,
                                   a.south_out, mo, &lk))
        return;
    finish_task<LC, false>(a, a.ms_out, tk, p, mo, lane);
}

// ---- persistent form ------------------------------------------------------

// Loads that bypass L1: data another SM wrote earlier in the same launch.
template <class T>
__device__ __forceinline__ T ld_cg(const T* p)
{
    static_assert(sizeof(T) % 8 == 0, "8-byte words");
    T v;
    auto* d = reinterpret_cast<unsigned long long*>(&v);
    auto* q = reinterpret_cast<const unsigned long long*>(p);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 8); ++i) d[i] = __ldcg(q + i);
    return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Generic-proxy stores of one step are read by the tensor memory
// accelerator (async proxy) in the next: a proxy fence on both sides of the
// barrier.
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// The first wait of the launch that gave up: kind (1: grid barrier, 2: a
// staged-row wait), step, CTA and two words of context.
__device__ __forceinline__ void record_wait(const PersistArgs& q, int kind, int j, int x, int y)
{
    if (atomicCAS(q.diag, 0, kind) == 0) {
        q.diag[1] = j;
        q.diag[2] = blockIdx.x;
        q.diag[3] = x;
        q.diag[4] = y;
        q.diag[5] = gridDim.x;
    }
}

// Plan of step j of scenario i (as batch_plan_kernel), by one thread.
__device__ __forceinline__ void plan_one(const PersistArgs& q, int i, int j, double t_stop)
{
    const BatchArgs& a = q.a;
    const int64_t k = q.k0 + j;
    const MemberClock* ms_in = q.ms + (k % 3) * q.S;
    MemberClock* ms_out = q.ms + ((k + 1) % 3) * q.S;
    MemberClock* ms_clr = q.ms + ((k + 2) % 3) * q.S;
    const ScenDesc sd = a.scen[i];
    const MemberClock in = ld_cg(ms_in + i);
    const double t_end = sd.t_end < t_stop ? sd.t_end : t_stop;
    const StepPlan sp = plan_step_p(a.alpha_dx, a.g, a.dt_cap, a.dt_fixed, a.h_floor, a.rain_block,
                                    t_end, sd.hyeto, sd.nb, sd.rain_mult, in);
    MemberPlan p;
    fill_plan(p, sp, a.g, a.dxd);
    p.cur = in.cur;
    p.ckpt = -1;
    p.q_in = 0.0f;
    ms_clr[i].hmax_bits = 0u;
    if (!sp.active) {
        ms_out[i] = in;
    } else {  // the maximum slot was cleared two steps ago: the step phase raises it
        ms_out[i].t = sp.t_next;
        ms_out[i].steps = in.steps + 1;
        ms_out[i].cur = 1 - in.cur;
        atomicAdd(a.rain_acc + i, (double)sp.dr * a.cell_area * sd.ncell);
        atomicOr(q.any_active + (j & 1), 1);
    }
    a.plan[i] = p;
}

// Grid-wide barrier of a cooperative launch with a bounded spin; the CTA
// that arrives last plans step j for every scenario (the previous step's
// maxima are complete by then) before it releases the others, unless j is
// past the launch's last step.  Returns false if this wait or an earlier one
// anywhere gave up.
__device__ __forceinline__ bool grid_barrier_plan(const PersistArgs& q, int j, double t_stop,
                                                  int* flag_s)
{
    const bool plan = j < q.max_steps;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nt = blockDim.x * blockDim.y;
    fence_proxy_async_global();
    __syncthreads();
    unsigned gen = 0;
    if (tid == 0) {
        __threadfence();
        gen = ld_acquire_u32(q.bar + 1);
        *flag_s = atomicAdd(q.bar, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    const bool last = *flag_s == 1;
    if (last && plan) {
        __threadfence();
        if (tid == 0) {  // both were last used two steps ago
            q.task_next[j & 1] = 0u;
            q.any_active[j & 1] = 0;
        }
        __syncthreads();
        for (int i = tid; i < q.S; i += nt) plan_one(q, i, j, t_stop);
        __syncthreads();
    }
    if (last && tid == 0) {
        atomicExch(q.bar, 0u);
        __threadfence();
        atomicAdd(q.bar + 1, 1u);
    }
    __syncthreads();
    if (tid == 0) {
        int ok = 1;
        if (!last) {
            const long long t0 = clock64();
            while (ld_acquire_u32(q.bar + 1) == gen) {
                if (clock64() - t0 > q.budget) {
                    atomicOr(q.a.err, 2);
                    record_wait(q, 1, j, (int)ld_acquire_u32(q.bar), (int)gen);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*reinterpret_cast<volatile const int*>(q.a.err) & 2) ok = 0;
        *flag_s = ok ? 2 : 3;
    }
    __syncthreads();
    fence_proxy_async_global();
    return *flag_s == 2;
}

// One warp task of the step phase (the batch_tma_kernel body, with the plan
// read past L1 and the volume slots updated atomically: a task may run on a
// different SM each step).
// Returns false if a wait of the march gave up (the warp then takes no
// further task: its barriers may still have a copy in flight).
template <int LIM, bool LC>
__device__ __forceinline__ bool persistent_task(const PersistArgs& q, int j, int t, MemberClock* ms_out,
                                                int lane, uint32_t bar0, unsigned char* my_stages)
{
    const BatchArgs& a = q.a;
    const WarpTask tk = a.tasks[t];
    const int i = tk.scen;
    const MemberPlan p = ld_cg(a.plan + i);
    if (!p.active) return true;
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
    float* dst = sd.state + (size_t)(1 - p.cur) * 3 * sd.plane;
    LandK lk;
    if (LC) lk = batch_land_k(a.scen + i, p.dr, p.dt, lane);
    MarchOut mo;
    const bool ok = tma_march<false, LC, LIM>(a.maps + 2 * i, a.maps + 2 * i + 1, p.cur * 3, bar0,
                                              my_stages, dst, nullptr, nullptr, a.err, sd.plane,
                                              sd.ny, sd.nx, sd.ld, tk.c0, tk.r0, tk.r1, lane, k,
                                              p.dt_dx, sd.scale, p.dr, a.east_out, a.south_out, mo,
                                              &lk);
    if (!ok) {
        if (lane == 0) record_wait(q, 2, j, t, i);
        return false;
    }
    // the warp's barriers and stages serve its next task: retire the barriers
    // (every copy has landed) and order the stages' generic reads before the
    // next task's copies overwrite them
    __syncwarp();
    if (lane == 0) {
        fence_proxy_async_smem();
        for (int s = 0; s < kTmaNS; ++s) mbar_inval(bar0 + 8u * s);
    }
    __syncwarp();
    finish_task<LC, true>(a, ms_out, tk, p, mo, lane);
    return true;
}

template <int W, int LIM, bool LC>
__global__ void __launch_bounds__(32 * W, 20 / W) batch_persistent_kernel(const __grid_constant__ PersistArgs q)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int flag_s;
    const BatchArgs& a = q.a;
    const int lane = threadIdx.x;
    const int w = threadIdx.y;
    const bool first_thread = blockIdx.x == 0 && w == 0 && lane == 0;
    uint32_t bar0;
    unsigned char* my_stages;
    tma_march_smem(smem_raw, W, w, bar0, my_stages);
    const double t_stop = *a.t_stop;
    int done = 0;
    if (grid_barrier_plan(q, 0, t_stop, &flag_s)) {  // plans step 0
        done = q.max_steps;
        for (int j = 0; j < q.max_steps; ++j) {
            if (__ldcg(q.any_active + (j & 1)) == 0) {  // every scenario has arrived
                done = j + 1;
                break;
            }
            const int64_t k = q.k0 + j;
            MemberClock* ms_out = q.ms + ((k + 1) % 3) * q.S;
            // step phase: warp w takes task w, then draws the tasks past the
            // first round from a counter (no burst of draws at the start)
            const unsigned nw = gridDim.x * W;
            unsigned t = blockIdx.x * W + w;
            while (t < (unsigned)a.ntasks) {
                if (!persistent_task<LIM, LC>(q, j, (int)t, ms_out, lane, bar0, my_stages)) break;
                if (nw >= (unsigned)a.ntasks) break;
                unsigned d = 0;
                if (lane == 0) d = atomicAdd(q.task_next + (j & 1), 1u);
                t = nw + __shfl_sync(0xffffffffu, d, 0);
            }
            if (!grid_barrier_plan(q, j + 1, t_stop, &flag_s)) {  // plans step j + 1
                done = j + 1;
                break;
            }
        }
    }
    if (first_thread) *q.steps_done = done;
}

}  // namespace

int batch_tma_prepare()
{
    cudaError_t e = cudaSuccess;
    for (auto f : {batch_tma_kernel<4, 0, false>, batch_tma_kernel<4, 1, false>,
                   batch_tma_kernel<4, 0, true>, batch_tma_kernel<4, 1, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma_march_smem_bytes(4));
    for (auto f : {batch_tma_kernel<8, 0, false>, batch_tma_kernel<8, 1, false>,
                   batch_tma_kernel<8, 0, true>, batch_tma_kernel<8, 1, true>})
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tma_march_smem_bytes(8));
    return e == cudaSuccess ? 0 : -1;
}

namespace {

template <int W, bool LC>
void launch_tma_w(const BatchArgs& a, cudaStream_t s)
{
    const unsigned g = (a.ntasks + W - 1) / W;
    if (a.limiter)
        batch_tma_kernel<W, 1, LC><<<g, dim3(32, W), tma_march_smem_bytes(W), s>>>(a);
    else
        batch_tma_kernel<W, 0, LC><<<g, dim3(32, W), tma_march_smem_bytes(W), s>>>(a);
}

}  // namespace

// the limiter and land cover are fixed at compile time (one instantiation
// per setting)
void launch_batch_step_tma(const BatchArgs& a, int warps_per_cta, cudaStream_t s)
{
    if (warps_per_cta >= 8)
        a.lc ? launch_tma_w<8, true>(a, s) : launch_tma_w<8, false>(a, s);
    else
        a.lc ? launch_tma_w<4, true>(a, s) : launch_tma_w<4, false>(a, s);
}

// One cooperative launch (its CTAs are resident together, which the grid
// barrier needs): as many CTAs of four warps as fit on the GPU.
cudaError_t launch_batch_persistent(const PersistArgs& q, cudaStream_t s)
{
    auto f = q.a.lc ? (q.a.limiter ? batch_persistent_kernel<4, 1, true> : batch_persistent_kernel<4, 0, true>)
                    : (q.a.limiter ? batch_persistent_kernel<4, 1, false> : batch_persistent_kernel<4, 0, false>);
    const size_t shm = tma_march_smem_bytes(4);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    int dev = 0, nsm = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, 128, shm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    void* args[] = {const_cast<PersistArgs*>(&q)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(f), dim3(nsm * per_sm),
                                       dim3(32, 4), args, shm, s);
}

void launch_batch_plan(const BatchArgs& a, int n_scen, cudaStream_t s)
{
    batch_plan_kernel<<<(n_scen + 127) / 128, 128, 0, s>>>(a, n_scen);
}

void launch_batch_step(const BatchArgs& a, int warps_per_cta, cudaStream_t s)
{
    if (warps_per_cta >= 8) {
        if (a.lc)
            batch_step_kernel<8, true><<<(a.ntasks + 7) / 8, dim3(32, 8), 0, s>>>(a);
        else
            batch_step_kernel<8, false><<<(a.ntasks + 7) / 8, dim3(32, 8), 0, s>>>(a);
    } else {
        if (a.lc)
            batch_step_kernel<4, true><<<(a.ntasks + 3) / 4, dim3(32, 4), 0, s>>>(a);
        else
            batch_step_kernel<4, false><<<(a.ntasks + 3) / 4, dim3(32, 4), 0, s>>>(a);
    }
}

}  // namespace flood
