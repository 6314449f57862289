// Inflow hydrograph boundary: a discharge series (one value per rain block,
// m^3/s) entering through the west-edge links of a segment of rows, spread
// evenly over them.  The per-step flux per unit width is part of each
// member's step plan (step_kernel.cu's plan kernel); the step kernels put it
// on the west links of those rows instead of the wall.
#include <cmath>
#include <vector>

#include "grid.cuh"

#define CK FLOOD_CK

extern "C" int flood_set_inflow(flood_grid* g, int r0, int r1, const float* series, int n_blocks)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (n_blocks == 0) {  // remove the boundary
        CK(g, cudaDeviceSynchronize());
        if (g->inflow) cudaFree(g->inflow);
        g->inflow = nullptr;
        g->inflow_blocks = g->in_r0 = g->in_r1 = 0;
        g->epoch++;
        return FLOOD_OK;
    }
    if (!series || n_blocks < 0 || r0 < 0 || r1 > g->ny || r0 >= r1)
        return flood::fail(g, FLOOD_ERR_ARG, "need 0 <= r0 < r1 <= ny and a series");
    std::vector<float> hs(n_blocks);
    CK(g, cudaMemcpy(hs.data(), series, sizeof(float) * n_blocks, cudaMemcpyDefault));
    for (float v : hs)
        if (!(v >= 0.0f) || !std::isfinite(v))
            return flood::fail(g, FLOOD_ERR_ARG, "discharges must be finite and >= 0");
    CK(g, cudaDeviceSynchronize());
    int rc = flood::dalloc(g, &g->inflow, n_blocks);
    if (rc) return rc;
    CK(g, cudaMemcpy(g->inflow, hs.data(), sizeof(float) * n_blocks, cudaMemcpyHostToDevice));
    g->inflow_blocks = n_blocks;
    g->in_r0 = r0;
    g->in_r1 = r1;
    g->epoch++;
    return FLOOD_OK;
}

extern "C" int flood_inflow_volume(flood_grid* g, double* volume)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (!g->M || !g->inflow_acc) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (!volume) return flood::fail(g, FLOOD_ERR_ARG, "volume is NULL");
    CK(g, cudaDeviceSynchronize());
    CK(g, cudaMemcpy(volume, g->inflow_acc, sizeof(double) * g->M, cudaMemcpyDeviceToHost));
    return FLOOD_OK;
}
