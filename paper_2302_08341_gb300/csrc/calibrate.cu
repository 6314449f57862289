// Gradient calibration (extension beyond the paper, whose uncertain inputs
// are estimated by the particle filter alone): a coarse multiplicative
// roughness field over the base Manning field, its gradient from the last
// flood_adjoint by the chain rule, and one clipped Polyak step in
// log-parameter space on the per-member rain multipliers and that field.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grid.cuh"

#define CK FLOOD_CK

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int kRedThreads = 256;
constexpr int kCalThreads = 1024;

// Fine index i lies in coarse block floor(i * cn / n); block k therefore
// starts at ceil(k * n / cn).
__device__ __forceinline__ int block_lo(int k, int n, int cn)
{
    return (int)(((long long)k * n + cn - 1) / cn);
}

// n(r, c) = n0(r, c) * f[block(r, c)], rounded once (FP32 product).
__global__ void apply_factor_kernel(const float* __restrict__ n0, const float* __restrict__ f,
                                    int ny, int nx, int ld, int cy, int cx, float* __restrict__ n)
{
    const size_t total = (size_t)ny * nx;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / nx), c = (int)(t % nx);
        const int br = (int)(((long long)r * cy) / ny), bc = (int)(((long long)c * cx) / nx);
        const size_t o = (size_t)r * ld + c;
        n[o] = __fmul_rn(n0[o], f[br * cx + bc]);
    }
}

// One CTA per coarse block: sum of n0 * dL/dn over the block's cells in FP64,
// each thread over a fixed subset, then a fixed shared-memory tree.
__global__ void __launch_bounds__(kRedThreads) factor_grad_kernel(
    const float* __restrict__ n0, int ld, const float* __restrict__ gn, int ny, int nx, int cy,
    int cx, double* __restrict__ out)
{
    const int b = blockIdx.x, br = b / cx, bc = b % cx;
    const int r0 = block_lo(br, ny, cy), r1 = block_lo(br + 1, ny, cy);
    const int c0 = block_lo(bc, nx, cx), c1 = block_lo(bc + 1, nx, cx);
    const int w = c1 - c0;
    const long long cnt = (long long)(r1 - r0) * w;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const int r = r0 + (int)(i / w), c = c0 + (int)(i % w);
        acc += (double)n0[(size_t)r * ld + c] * (double)gn[(size_t)r * nx + c];
    }
    __shared__ double red[kRedThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[b] = red[0];
}

struct CalArgs {
    const float* y;        // [ns][M][G] gauge outputs recorded by the adjoint
    const double* d;       // [ns][G] observations
    const double* gpart;   // [M][nslot][2] per-warp dL/d(rain multiplier), dL/d(scale)
    float* rain_mult;      // [M] in / out
    double* loss;          // [M] out
    double* rain_grad;     // [M] out: dL_i/d(rain multiplier), for the joint step (land cover)
    int joint;             // 1: the rain multiplier moves in the joint land-cover step instead
    float* fac;            // [B] in / out (or null)
    const double* fgrad;   // [B]
    int ns, G, M, nslot, B;
    double eta, delta;
};

__device__ __forceinline__ double clip(double x, double d) { return fmin(fmax(x, -d), d); }

// Single CTA: per-member loss and rain step (with land cover only the loss
// and the rain gradient: the joint step takes the rain multiplier with the
// land-cover parameters), then the field step (its squared gradient norm by
// a fixed-order tree).
__global__ void __launch_bounds__(kCalThreads) calib_kernel(const CalArgs a)
{
    for (int m = threadIdx.x; m < a.M; m += blockDim.x) {
        double L = 0.0;
        for (int si = 0; si < a.ns; ++si)
            for (int k = 0; k < a.G; ++k) {
                const double e = __dsub_rn((double)a.y[((size_t)si * a.M + m) * a.G + k],
                                           a.d[(size_t)si * a.G + k]);
                L = __dadd_rn(L, __dmul_rn(e, e));
            }
        a.loss[m] = L;
        double gm = 0.0;  // the same order as the rain gradient flood_adjoint reports
        for (int k = 0; k < a.nslot; ++k) gm += a.gpart[((size_t)m * a.nslot + k) * 2];
        if (a.joint) {
            a.rain_grad[m] = gm;
            continue;
        }
        const double mi = (double)a.rain_mult[m];
        const double gt = mi * gm;
        const double st = gt != 0.0 ? clip(-a.eta * L / gt, a.delta) : 0.0;
        a.rain_mult[m] = (float)(mi * exp(st));
    }
    if (a.B == 0) return;  // the same for every thread of the CTA
    __shared__ double red[kCalThreads];
    __shared__ double s_L;
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0;
        for (int m = 0; m < a.M; ++m) L += a.loss[m];
        s_L = L;
    }
    double acc = 0.0;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        const double G = (double)a.fac[b] * a.fgrad[b];
        acc += G * G;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kCalThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double s2 = red[0], L = s_L;
    for (int b = threadIdx.x; b < a.B; b += blockDim.x) {
        const double f = (double)a.fac[b];
        const double G = f * a.fgrad[b];
        const double st = s2 > 0.0 ? clip(-a.eta * L * G / s2, a.delta) : 0.0;
        a.fac[b] = (float)(f * exp(st));
    }
}

void launch_apply(flood_grid* g, cudaStream_t s)
{
    const size_t total = (size_t)g->ny * g->nx;
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 4096);
    apply_factor_kernel<<<blocks, 256, 0, s>>>(g->n0, g->fac, g->ny, g->nx, g->ld, g->fcy, g->fcx,
                                               g->n);
    g->launches++;
}

// The adjoint's gradients still describe the ensemble as it is now.
int check_fresh_adjoint(flood_grid* g, bool need_gn)
{
    if (g->adj_epoch != g->epoch)
        return flood::fail(g, FLOOD_ERR_STATE,
                           "no flood_adjoint since the ensemble last changed (or its step was spent)");
    if (need_gn && (!g->adj_gn || !g->gn_out))
        return flood::fail(g, FLOOD_ERR_STATE, "the last flood_adjoint was not given grad_n");
    return FLOOD_OK;
}

}  // namespace

extern "C" int flood_set_roughness_factor(flood_grid* g, int cy, int cx, const float* f,
                                          void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->lc_on)
        return flood::fail(g, FLOOD_ERR_STATE, "with land cover the roughness comes from the classes");
    if (!f || cy < 1 || cx < 1 || cy > g->ny || cx > g->nx)
        return flood::fail(g, FLOOD_ERR_ARG, "need f and 1 <= cy <= ny, 1 <= cx <= nx");
    std::vector<float> hf((size_t)cy * cx);
    CK(g, cudaMemcpy(hf.data(), f, sizeof(float) * hf.size(), cudaMemcpyDefault));
    for (float v : hf)
        if (!(v > 0.0f) || !std::isfinite(v))
            return flood::fail(g, FLOOD_ERR_ARG, "factor values must be positive and finite");
    cudaStream_t s = S(stream);
    CK(g, cudaStreamSynchronize(s));
    int rc;
    if (!g->n0) {
        if ((rc = flood::dalloc(g, &g->n0, g->plane))) return rc;
        CK(g, cudaMemcpy(g->n0, g->n, sizeof(float) * g->plane, cudaMemcpyDeviceToDevice));
    }
    if (!g->fac || cy != g->fcy || cx != g->fcx) {
        if ((rc = flood::dalloc(g, &g->fac, hf.size()))) return rc;
        if ((rc = flood::dalloc(g, &g->fgrad, hf.size()))) return rc;
        g->fcy = cy;
        g->fcx = cx;
    }
    CK(g, cudaMemcpy(g->fac, hf.data(), sizeof(float) * hf.size(), cudaMemcpyHostToDevice));
    launch_apply(g, s);
    CK(g, cudaGetLastError());
    CK(g, cudaStreamSynchronize(s));
    g->epoch++;
    return FLOOD_OK;
}

extern "C" int flood_get_roughness_factor(flood_grid* g, int* cy, int* cx, float* f)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->fac) return flood::fail(g, FLOOD_ERR_STATE, "no roughness factor field has been set");
    if (cy) *cy = g->fcy;
    if (cx) *cx = g->fcx;
    if (f) CK(g, cudaMemcpy(f, g->fac, sizeof(float) * g->fcy * g->fcx, cudaMemcpyDefault));
    return FLOOD_OK;
}

extern "C" int flood_roughness_factor_grad(flood_grid* g, double* grad, void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!grad) return flood::fail(g, FLOOD_ERR_ARG, "grad is NULL");
    if (!g->fac) return flood::fail(g, FLOOD_ERR_STATE, "no roughness factor field has been set");
    int rc = check_fresh_adjoint(g, true);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    factor_grad_kernel<<<g->fcy * g->fcx, kRedThreads, 0, s>>>(g->n0, g->ld, g->gn_out, g->ny,
                                                               g->nx, g->fcy, g->fcx, g->fgrad);
    g->launches++;
    CK(g, cudaGetLastError());
    CK(g, cudaMemcpyAsync(grad, g->fgrad, sizeof(double) * g->fcy * g->fcx, cudaMemcpyDefault, s));
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}

extern "C" int flood_calibration_step(flood_grid* g, double eta, double delta, double* loss_out,
                                      void* stream)
{
    const flood::TraceRange range("flood_calibration_step");
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!(eta > 0.0) || !(delta > 0.0))
        return flood::fail(g, FLOOD_ERR_ARG, "eta and delta must be positive");
    if (g->M == 0) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    const bool field = g->fac != nullptr;
    int rc = check_fresh_adjoint(g, field);
    if (rc) return rc;
    cudaStream_t s = S(stream);
    if (g->closs_cap < g->M) {
        if ((rc = flood::dalloc(g, &g->closs, 2 * (size_t)g->M))) return rc;
        g->closs_cap = g->M;
    }
    if (field) {
        factor_grad_kernel<<<g->fcy * g->fcx, kRedThreads, 0, s>>>(
            g->n0, g->ld, g->gn_out, g->ny, g->nx, g->fcy, g->fcx, g->fgrad);
        g->launches++;
    }
    CalArgs a{};
    a.y = g->samp_y;
    a.d = g->samp_d;
    a.gpart = g->gpart;
    a.rain_mult = g->rain_mult;
    a.loss = g->closs;
    a.rain_grad = g->closs + g->M;
    a.joint = g->lc_on ? 1 : 0;
    a.fac = g->fac;
    a.fgrad = g->fgrad;
    a.ns = g->adj_ns;
    a.G = g->adj_G;
    a.M = g->M;
    a.nslot = g->adj_nslot;
    a.B = field ? g->fcy * g->fcx : 0;
    a.eta = eta;
    a.delta = delta;
    calib_kernel<<<1, kCalThreads, 0, s>>>(a);
    g->launches++;
    if (field) launch_apply(g, s);
    CK(g, cudaGetLastError());
    if (g->lc_on && (rc = flood::land_calibration_step(g, g->closs, g->closs + g->M, eta, delta, s)))
        return rc;
    if (loss_out)
        CK(g, cudaMemcpyAsync(loss_out, g->closs, sizeof(double) * g->M, cudaMemcpyDefault, s));
    CK(g, cudaStreamSynchronize(s));
    g->epoch++;  // the gradients are spent
    return FLOOD_OK;
}
