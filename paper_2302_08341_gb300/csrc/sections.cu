// Streamflow gauges (Section 4.1 / 4.4 observe stream gauges next to depth
// gauges): the discharge of every member through straight sections of
// links, Q = sum of q dx over the section (Eq. 5's link discharges),
// positive toward increasing index.  Together with a relative observation
// error (pf_assimilate's sigma_rel, or per-gauge sigma = alpha * d, Section
// 4.4) these are the particle filter's flow observations.
#include <vector>

#include "grid.cuh"

#define CK FLOOD_CK

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

struct SecDev {
    int axis, fixed, start, end;
};

// One warp per (member, section): lanes take the links in a fixed stride,
// FP64 sums, then a fixed shuffle tree.
__global__ void flow_kernel(const float* __restrict__ state, const flood::MemberClock* __restrict__ ms,
                            const SecDev* __restrict__ sec, int n_sec, int M, int ld, size_t plane,
                            double dx, float* __restrict__ out)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= M * n_sec) return;  // whole warps
    const int m = w / n_sec, k = w % n_sec;
    const SecDev s = sec[k];
    const float* base = state + (size_t)(ms[m].cur * M + m) * 3 * plane;
    const float* q = base + (s.axis == 0 ? plane : 2 * plane);
    double acc = 0.0;
    for (int i = s.start + lane; i < s.end; i += 32) {
        const size_t o = s.axis == 0 ? (size_t)i * ld + s.fixed : (size_t)s.fixed * ld + i;
        acc += (double)q[o];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) out[(size_t)m * n_sec + k] = (float)(acc * dx);
}

}  // namespace

extern "C" int flood_flow_sample(flood_grid* g, int n_sections, const flood_section* sections,
                                 float* q_out, void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (n_sections < 1 || !sections || !q_out)
        return flood::fail(g, FLOOD_ERR_ARG, "need sections and q_out");
    std::vector<SecDev> sd(n_sections);
    for (int k = 0; k < n_sections; ++k) {
        const flood_section& s = sections[k];
        const int along = s.axis == 0 ? g->ny : g->nx, across = s.axis == 0 ? g->nx : g->ny;
        if ((s.axis != 0 && s.axis != 1) || s.fixed < 0 || s.fixed >= across || s.start < 0 ||
            s.end > along || s.start >= s.end)
            return flood::fail(g, FLOOD_ERR_ARG, "section outside the grid");
        sd[k] = {s.axis, s.fixed, s.start, s.end};
    }
    cudaStream_t st = S(stream);
    SecDev* dsec = nullptr;
    float* dout = nullptr;
    const size_t nout = (size_t)g->M * n_sections;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dsec), sizeof(SecDev) * n_sections, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&dout), sizeof(float) * nout, st);
    if (e != cudaSuccess)
        return flood::fail(g, e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA,
                           std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    CK(g, cudaMemcpyAsync(dsec, sd.data(), sizeof(SecDev) * n_sections, cudaMemcpyHostToDevice, st));
    const size_t threads = nout * 32;
    flow_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        g->state, g->ms + (g->k % 3) * g->M, dsec, n_sections, g->M, g->ld, g->plane, g->p.dx, dout);
    g->launches++;
    CK(g, cudaGetLastError());
    CK(g, cudaMemcpyAsync(q_out, dout, sizeof(float) * nout, cudaMemcpyDefault, st));
    CK(g, cudaFreeAsync(dsec, st));
    CK(g, cudaFreeAsync(dout, st));
    CK(g, cudaStreamSynchronize(st));
    return FLOOD_OK;
}
