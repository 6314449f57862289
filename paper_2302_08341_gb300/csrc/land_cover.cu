// Land cover (Section 4.1, Table 1): a class per cell, with per-class runoff
// coefficient (the share of the rain that stays on the surface), drainage
// (the drainage capacity of the pipe network on hardened ground) and Manning
// n, and cells outside the domain.  The class's roughness and the drainage
// rate are the per-member uncertain inputs of the paper's ensemble; they
// follow their particle through a resampling.
//
// Cells outside the domain get a bed out of reach (kWallZ) and no rain, so
// Eq. 3 gives every link into them a zero flow depth: they never get wet and
// nothing crosses them.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grid.cuh"
#include "pf_kernels.cuh"
#include "tma.cuh"

#define CK FLOOD_CK

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr float kWallZ = 1.0e6f;  // m: a bed no water level reaches
constexpr int kMaxClasses = 4;

// After a resampling, slot s takes particle src[s]'s parameters (one CTA).
__global__ void land_permute_kernel(float* __restrict__ lc_n, float* __restrict__ lc_drain,
                                    const int32_t* __restrict__ src,
                                    const int32_t* __restrict__ resampled, int M)
{
    if (!*resampled) return;
    extern __shared__ float old[];  // [M][4] then [M]
    for (int i = threadIdx.x; i < M * 4; i += blockDim.x) old[i] = lc_n[i];
    for (int i = threadIdx.x; i < M; i += blockDim.x) old[M * 4 + i] = lc_drain[i];
    __syncthreads();
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
        const int p = src[s];
        for (int q = 0; q < 4; ++q) lc_n[s * 4 + q] = old[p * 4 + q];
        lc_drain[s] = old[M * 4 + p];
    }
}

// The reverse pass's land-cover fields (one thread per cell of the padded
// plane): plane 0 the bed, plane 1 + m member m's Manning n (its class's, as
// the step looks it up), plane M + 1 the share of the rain that stays, plane
// M + 2 the drainage flag.
__global__ void land_adjoint_fields_kernel(float* __restrict__ out, const float* __restrict__ z,
                                           const uint8_t* __restrict__ cls,
                                           const float* __restrict__ lc_n, float4 runoff,
                                           float4 drains, int M, size_t plane)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = cls[i];
        out[i] = z[i];
        for (int m = 0; m < M; ++m) out[(size_t)(1 + m) * plane + i] = lc_n[(size_t)m * 4 + k];
        out[(size_t)(M + 1) * plane + i] =
            k == 0 ? runoff.x : k == 1 ? runoff.y : k == 2 ? runoff.z : runoff.w;
        out[(size_t)(M + 2) * plane + i] =
            k == 0 ? drains.x : k == 1 ? drains.y : k == 2 ? drains.z : drains.w;
    }
}

// dL_m/dn of each class for member m (one CTA per member): the per-cell
// Manning gradients of the member summed over the cells of each class, in
// FP64 and a fixed order (deterministic).
constexpr int kGradThreads = 256;

__global__ void __launch_bounds__(kGradThreads) land_class_grad_kernel(
    const float* __restrict__ gnm, const uint8_t* __restrict__ cls, int ny, int nx, int ld,
    size_t plane, double* __restrict__ out)
{
    const int m = blockIdx.x;
    const float* g = gnm + (size_t)m * plane;
    double acc[kMaxClasses] = {0.0, 0.0, 0.0, 0.0};
    const size_t cells = (size_t)ny * nx;
    for (size_t i = threadIdx.x; i < cells; i += kGradThreads) {
        const size_t o = (i / nx) * ld + i % nx;
        const double v = g[o];
        const int k = cls[o];
#pragma unroll
        for (int q = 0; q < kMaxClasses; ++q) acc[q] += (k == q) ? v : 0.0;
    }
    __shared__ double red[kMaxClasses][kGradThreads];
#pragma unroll
    for (int q = 0; q < kMaxClasses; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kGradThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < kMaxClasses; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < kMaxClasses) out[(size_t)m * kMaxClasses + threadIdx.x] = red[threadIdx.x][0];
}

// Cells of the classes in `mask` (outside the domain) hold no water and no
// flow: zero h, qx, qy there in both buffers of members [m0, m0 + count).
__global__ void zero_outside_kernel(float* __restrict__ state, const uint8_t* __restrict__ cls,
                                    unsigned mask, int M, int m0, int count, size_t plane)
{
    const size_t total = (size_t)2 * count * plane;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t e = t % plane;
        if (!((mask >> cls[e]) & 1u)) continue;
        const size_t k = t / plane;              // (buffer, member) pair
        const int b = (int)(k / count), m = m0 + (int)(k % count);
        float* base = state + ((size_t)b * M + m) * 3 * plane;
        base[e] = 0.0f;
        base[plane + e] = 0.0f;
        base[2 * plane + e] = 0.0f;
    }
}

}  // namespace

namespace flood {

void land_zero_outside(flood_grid* g, int m0, int count, cudaStream_t s)
{
    if (!g->lc_out_mask || count < 1) return;
    zero_outside_kernel<<<g->n_sm * 4, 256, 0, s>>>(g->state, g->cls8, g->lc_out_mask, g->M, m0,
                                                    count, g->plane);
    g->launches++;
}

int land_tiles(flood_grid* g)
{
    const int spans = (g->nx + 127) / 128, R = g->rows_per_strip;
    const int strips = (g->ny + R - 1) / R;
    std::vector<int2> t;
    t.reserve((size_t)spans * strips);
    for (int st = 0; st < strips; ++st)
        for (int sp = 0; sp < spans; ++sp) {
            bool inside = false;
            for (int r = st * R; r < std::min(g->ny, (st + 1) * R) && !inside; ++r)
                inside = !g->lc_span_out[(size_t)r * spans + sp];
            if (inside) t.push_back(make_int2(sp, st));
        }
    if (t.empty()) t.push_back(make_int2(0, 0));  // a grid wholly outside: one idle tile
    int rc = dalloc(g, &g->tiles, t.size());
    if (rc) return rc;
    CK(g, cudaMemcpy(g->tiles, t.data(), sizeof(int2) * t.size(), cudaMemcpyHostToDevice));
    g->n_tiles = (int)t.size();
    g->tiles_rows = R;
    return FLOOD_OK;
}

// One joint step per member over all of its parameters -- the rain
// multiplier, the class roughness and the drainage rate -- in log-parameter
// space with the Polyak length of its own loss: G = theta * dL/dtheta,
// step = clip(-eta L G / |G|^2, delta); no step where |G| = 0.  One step for
// the whole vector removes eta L to first order (a rain step beside a
// land-cover step would remove it twice).  cgrad may be null (no per-cell
// Manning gradients): the class roughness then stays.
__global__ void land_calib_kernel(float* __restrict__ rain_mult, float* __restrict__ lc_n,
                                  float* __restrict__ lc_drain, const double* __restrict__ rgrad,
                                  const double* __restrict__ cgrad, const double* __restrict__ dgrad,
                                  const double* __restrict__ loss, int M, int K, double eta,
                                  double delta)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double G[kMaxClasses + 2], s2 = 0.0;
    for (int q = 0; q < K; ++q) {
        G[q] = cgrad ? (double)lc_n[(size_t)m * 4 + q] * cgrad[(size_t)m * kMaxClasses + q] : 0.0;
        s2 += G[q] * G[q];
    }
    G[K] = (double)lc_drain[m] * dgrad[m];
    s2 += G[K] * G[K];
    G[K + 1] = (double)rain_mult[m] * rgrad[m];
    s2 += G[K + 1] * G[K + 1];
    if (!(s2 > 0.0)) return;
    const double c = -eta * loss[m] / s2;
    for (int q = 0; q < K; ++q) {
        const double n = (double)lc_n[(size_t)m * 4 + q];
        lc_n[(size_t)m * 4 + q] = (float)(n * exp(fmin(fmax(c * G[q], -delta), delta)));
    }
    const double d = (double)lc_drain[m];
    lc_drain[m] = (float)(d * exp(fmin(fmax(c * G[K], -delta), delta)));
    const double r = (double)rain_mult[m];
    rain_mult[m] = (float)(r * exp(fmin(fmax(c * G[K + 1], -delta), delta)));
}

int land_calibration_step(flood_grid* g, const double* loss, const double* rain_grad, double eta,
                          double delta, cudaStream_t s)
{
    const int M = g->M;
    const bool classes = g->adj_gn && g->gnm;
    if (classes && !g->lc_cgrad) {
        const int rc = dalloc(g, &g->lc_cgrad, (size_t)M * kMaxClasses);
        if (rc) return rc;
    }
    if (!g->lc_dgrad) {
        const int rc = dalloc(g, &g->lc_dgrad, (size_t)M);
        if (rc) return rc;
    }
    if (classes) {
        land_class_grad_kernel<<<M, kGradThreads, 0, s>>>(g->gnm, g->cls8, g->ny, g->nx, g->ld,
                                                          g->plane, g->lc_cgrad);
        g->launches++;
    }
    CK(g, cudaMemcpyAsync(g->lc_dgrad, g->adj_gdrain.data(), sizeof(double) * M,
                          cudaMemcpyHostToDevice, s));
    land_calib_kernel<<<(M + 127) / 128, 128, 0, s>>>(g->rain_mult, g->lc_n, g->lc_drain, rain_grad,
                                                      classes ? g->lc_cgrad : nullptr, g->lc_dgrad,
                                                      loss, M, g->lc_K, eta, delta);
    g->launches++;
    CK(g, cudaGetLastError());
    return FLOOD_OK;
}

int land_adjoint_fields(flood_grid* g, cudaStream_t s)
{
    const int M = g->M;
    if (!g->lc_adj) {
        const int rc = dalloc(g, &g->lc_adj, (size_t)(M + 3) * g->plane);
        if (rc) return rc;
    }
    const float4 ro = make_float4(g->lc_runoff[0], g->lc_runoff[1], g->lc_runoff[2], g->lc_runoff[3]);
    const float4 dr = make_float4(g->lc_drains[0], g->lc_drains[1], g->lc_drains[2], g->lc_drains[3]);
    const unsigned blocks = (unsigned)std::min<size_t>((g->plane + 255) / 256, 4096);
    land_adjoint_fields_kernel<<<blocks, 256, 0, s>>>(g->lc_adj, g->z, g->cls8, g->lc_n, ro, dr, M,
                                                      g->plane);
    g->launches++;
    CK(g, cudaGetLastError());
    return FLOOD_OK;
}

void launch_land_permute(float* lc_n, float* lc_drain, const int32_t* src, const int32_t* resampled,
                         int M, cudaStream_t s)
{
    land_permute_kernel<<<1, 256, sizeof(float) * 5 * M, s>>>(lc_n, lc_drain, src, resampled, M);
}

// Per-member defaults after flood_ensemble_init: the classes' own n, no
// drainage; drained volume cleared.
int land_ensemble_init(flood_grid* g)
{
    const int M = g->M;
    int rc;
    if ((rc = dalloc(g, &g->lc_n, (size_t)M * 4)) || (rc = dalloc(g, &g->lc_drain, M)) ||
        (rc = dalloc(g, &g->dacc, (size_t)M * g->nslot)))
        return rc;
    std::vector<float> n((size_t)M * 4);
    for (int m = 0; m < M; ++m)
        for (int q = 0; q < 4; ++q) n[(size_t)m * 4 + q] = g->lc_n0[q];
    std::vector<float> d(M, 0.0f);
    FLOOD_CK(g, cudaMemcpy(g->lc_n, n.data(), sizeof(float) * n.size(), cudaMemcpyHostToDevice));
    FLOOD_CK(g, cudaMemcpy(g->lc_drain, d.data(), sizeof(float) * M, cudaMemcpyHostToDevice));
    FLOOD_CK(g, cudaMemset(g->dacc, 0, sizeof(double) * M * g->nslot));
    if (g->lc_out_mask) {
        // cells outside the domain start dry and at rest (the step leaves
        // the tiles wholly outside it untouched); Eq. 4's maximum depth is
        // taken again without them
        land_zero_outside(g, 0, M, 0);
        MemberClock* slot = g->ms + (g->k % 3) * M;
        std::vector<MemberClock> c(M);
        FLOOD_CK(g, cudaMemcpy(c.data(), slot, sizeof(MemberClock) * M, cudaMemcpyDeviceToHost));
        for (auto& x : c) x.hmax_bits = 0;
        FLOOD_CK(g, cudaMemcpy(slot, c.data(), sizeof(MemberClock) * M, cudaMemcpyHostToDevice));
        launch_hmax(g->state, slot, M, g->ny, g->nx, g->ld, g->plane, g->n_sm, 0);
        g->launches++;
        FLOOD_CK(g, cudaGetLastError());
        FLOOD_CK(g, cudaDeviceSynchronize());
    }
    return FLOOD_OK;
}

}  // namespace flood

extern "C" int flood_set_land_cover(flood_grid* g, const uint8_t* cls, int n_classes,
                                    const flood_land_class* classes)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->lc_on) return flood::fail(g, FLOOD_ERR_STATE, "land cover is already set");
    if (g->fac)
        return flood::fail(g, FLOOD_ERR_STATE, "a roughness factor field is set: land cover replaces it");
    if (!cls || !classes || n_classes < 1 || n_classes > kMaxClasses)
        return flood::fail(g, FLOOD_ERR_ARG, "need cls, 1..4 classes and their table");
    for (int q = 0; q < n_classes; ++q) {
        const flood_land_class& k = classes[q];
        if (!(k.n > 0.0f) || !(k.runoff >= 0.0f && k.runoff <= 1.0f) ||
            (k.drains != 0 && k.drains != 1) || (k.outside != 0 && k.outside != 1))
            return flood::fail(g, FLOOD_ERR_ARG, "class needs n > 0, runoff in [0, 1], flags 0/1");
    }
    const size_t cells = (size_t)g->ny * g->nx;
    std::vector<uint8_t> hc(cells);
    CK(g, cudaMemcpy(hc.data(), cls, cells, cudaMemcpyDefault));
    std::vector<float> runoff(kMaxClasses, 1.0f), drains(kMaxClasses, 0.0f), n0(kMaxClasses, 0.05f);
    for (int q = 0; q < n_classes; ++q) {
        runoff[q] = classes[q].outside ? 0.0f : classes[q].runoff;
        drains[q] = classes[q].outside ? 0.0f : (float)classes[q].drains;
        n0[q] = classes[q].n;
    }
    double rain_cells = 0.0;
    std::vector<uint8_t> pad((size_t)g->ny * g->ld, 0);
    bool any_outside = false;
    for (int r = 0; r < g->ny; ++r)
        for (int c = 0; c < g->nx; ++c) {
            const uint8_t k = hc[(size_t)r * g->nx + c];
            if (k >= n_classes) return flood::fail(g, FLOOD_ERR_ARG, "class index out of range");
            pad[(size_t)r * g->ld + c] = k;
            rain_cells += runoff[k];
            any_outside |= classes[k].outside != 0;
        }
    // the bed of cells outside the domain moves out of reach
    if (any_outside) {
        std::vector<float> z(g->plane);
        CK(g, cudaMemcpy(z.data(), g->z, sizeof(float) * g->plane, cudaMemcpyDeviceToHost));
        for (int r = 0; r < g->ny; ++r)
            for (int c = 0; c < g->nx; ++c)
                if (classes[hc[(size_t)r * g->nx + c]].outside) z[(size_t)r * g->ld + c] = kWallZ;
        CK(g, cudaMemcpy(g->z, z.data(), sizeof(float) * g->plane, cudaMemcpyHostToDevice));
    }
    int rc = flood::dalloc(g, &g->cls8, pad.size());
    if (rc) return rc;
    // the TMA step's static planes with land cover: the bed (raised outside
    // the domain) and each cell's class code, where the roughness plane
    // would be (the roughness comes from the class)
    if ((rc = flood::dalloc(g, &g->zc, 2 * g->plane))) return rc;
    CK(g, cudaMemcpy(g->zc, g->z, sizeof(float) * g->plane, cudaMemcpyDeviceToDevice));
    {
        std::vector<uint32_t> codes(g->plane, 0u);
        for (size_t i = 0; i < g->plane; ++i) codes[i] = pad[i];
        CK(g, cudaMemcpy(g->zc + g->plane, codes.data(), sizeof(uint32_t) * g->plane,
                         cudaMemcpyHostToDevice));
    }
    if (flood::encode_map_3d(&g->static_map_lc, g->zc, g->ld, g->ny, 2, sizeof(float) * g->ld,
                             sizeof(float) * g->plane, flood::tma_box_cols(), 1, 2) != 0)
        return flood::fail(g, FLOOD_ERR_CUDA, "tensor map of the bed and class codes");
    CK(g, cudaMemcpy(g->cls8, pad.data(), pad.size(), cudaMemcpyHostToDevice));
    for (int q = 0; q < kMaxClasses; ++q) {
        g->lc_runoff[q] = runoff[q];
        g->lc_drains[q] = drains[q];
        g->lc_n0[q] = n0[q];
    }
    g->lc_out_mask = 0;
    for (int q = 0; q < n_classes; ++q)
        if (classes[q].outside) g->lc_out_mask |= (uint8_t)(1u << q);
    const int spans = (g->nx + 127) / 128;
    g->lc_span_out.assign((size_t)g->ny * spans, 1);
    for (int r = 0; r < g->ny; ++r)
        for (int c = 0; c < g->nx; ++c)
            if (!classes[hc[(size_t)r * g->nx + c]].outside) g->lc_span_out[(size_t)r * spans + c / 128] = 0;
    g->tiles_rows = 0;
    g->lc_K = n_classes;
    g->lc_rain_cells = rain_cells;
    g->lc_on = true;
    g->epoch++;
    if (g->M && (rc = flood::land_ensemble_init(g))) return rc;
    return FLOOD_OK;
}

extern "C" int flood_set_land_params(flood_grid* g, const float* n_class, const float* drain_rate)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->lc_on || !g->M) return flood::fail(g, FLOOD_ERR_STATE, "needs land cover and an ensemble");
    const int M = g->M, K = g->lc_K;
    CK(g, cudaDeviceSynchronize());
    if (n_class) {
        std::vector<float> in((size_t)M * K), n((size_t)M * 4);
        CK(g, cudaMemcpy(in.data(), n_class, sizeof(float) * in.size(), cudaMemcpyDefault));
        for (int m = 0; m < M; ++m)
            for (int q = 0; q < 4; ++q) {
                const float v = q < K ? in[(size_t)m * K + q] : g->lc_n0[q];
                if (!(v > 0.0f) || !std::isfinite(v))
                    return flood::fail(g, FLOOD_ERR_ARG, "class roughness must be positive");
                n[(size_t)m * 4 + q] = v;
            }
        CK(g, cudaMemcpy(g->lc_n, n.data(), sizeof(float) * n.size(), cudaMemcpyHostToDevice));
    }
    if (drain_rate) {
        std::vector<float> d(M);
        CK(g, cudaMemcpy(d.data(), drain_rate, sizeof(float) * M, cudaMemcpyDefault));
        for (float v : d)
            if (!(v >= 0.0f) || !std::isfinite(v))
                return flood::fail(g, FLOOD_ERR_ARG, "drainage rates must be >= 0");
        CK(g, cudaMemcpy(g->lc_drain, d.data(), sizeof(float) * M, cudaMemcpyHostToDevice));
    }
    g->epoch++;
    return FLOOD_OK;
}

extern "C" int flood_get_land_params(flood_grid* g, float* n_class, float* drain_rate)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->lc_on || !g->M) return flood::fail(g, FLOOD_ERR_STATE, "needs land cover and an ensemble");
    const int M = g->M, K = g->lc_K;
    CK(g, cudaDeviceSynchronize());
    if (n_class) {
        std::vector<float> n((size_t)M * 4), out((size_t)M * K);
        CK(g, cudaMemcpy(n.data(), g->lc_n, sizeof(float) * n.size(), cudaMemcpyDeviceToHost));
        for (int m = 0; m < M; ++m)
            for (int q = 0; q < K; ++q) out[(size_t)m * K + q] = n[(size_t)m * 4 + q];
        CK(g, cudaMemcpy(n_class, out.data(), sizeof(float) * out.size(), cudaMemcpyDefault));
    }
    if (drain_rate) CK(g, cudaMemcpy(drain_rate, g->lc_drain, sizeof(float) * M, cudaMemcpyDefault));
    return FLOOD_OK;
}

extern "C" int flood_drained_volume(flood_grid* g, double* drained)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->M) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (!drained) return flood::fail(g, FLOOD_ERR_ARG, "drained is NULL");
    const int M = g->M;
    if (!g->dacc) {
        std::fill(drained, drained + M, 0.0);
        return FLOOD_OK;
    }
    CK(g, cudaDeviceSynchronize());
    std::vector<double> d((size_t)M * g->nslot);
    CK(g, cudaMemcpy(d.data(), g->dacc, sizeof(double) * d.size(), cudaMemcpyDeviceToHost));
    for (int m = 0; m < M; ++m) {
        double acc = 0.0;
        for (int k = 0; k < g->nslot; ++k) acc += d[(size_t)m * g->nslot + k];
        drained[m] = acc;
    }
    return FLOOD_OK;
}

extern "C" int flood_adjoint_land_grad(flood_grid* g, double* grad_n_class, double* grad_drain,
                                       void* stream)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->lc_on) return flood::fail(g, FLOOD_ERR_STATE, "no land cover is set");
    if (g->adj_epoch != g->epoch || (int)g->adj_gdrain.size() != g->M)
        return flood::fail(g, FLOOD_ERR_STATE,
                           "no flood_adjoint since the ensemble last changed (or its step was spent)");
    const int M = g->M, K = g->lc_K;
    if (grad_drain) std::copy(g->adj_gdrain.begin(), g->adj_gdrain.end(), grad_drain);
    if (!grad_n_class) return FLOOD_OK;
    if (!g->adj_gn || !g->gnm)
        return flood::fail(g, FLOOD_ERR_STATE, "the last flood_adjoint was not given grad_n");
    cudaStream_t s = S(stream);
    if (!g->lc_cgrad) {
        const int rc = flood::dalloc(g, &g->lc_cgrad, (size_t)M * kMaxClasses);
        if (rc) return rc;
    }
    land_class_grad_kernel<<<M, kGradThreads, 0, s>>>(g->gnm, g->cls8, g->ny, g->nx, g->ld, g->plane,
                                                      g->lc_cgrad);
    g->launches++;
    CK(g, cudaGetLastError());
    std::vector<double> h((size_t)M * kMaxClasses);
    CK(g, cudaMemcpyAsync(h.data(), g->lc_cgrad, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    CK(g, cudaStreamSynchronize(s));
    for (int m = 0; m < M; ++m)
        for (int q = 0; q < K; ++q) grad_n_class[(size_t)m * K + q] = h[(size_t)m * kMaxClasses + q];
    return FLOOD_OK;
}
