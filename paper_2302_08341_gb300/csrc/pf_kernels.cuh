// Launchers of the particle-filter and reduction kernels (pf_kernels.cu).
#pragma once

#include "flood_internal.cuh"

namespace flood {

struct PfArgs {
    const float* y;        // [M][G] model outputs
    const double* d;       // [G] observations
    const double* sigma;   // [G] observation standard deviations
    double sigma_rel;      // > 0: sigma = sigma_rel * d
    double n_thr_frac;     // resample when N_eff < n_thr_frac * M
    int force;
    double u;              // systematic resampling draw in [0,1)
    const float* beta;     // [M] rain perturbation factors
    double* w;             // [M] weights (prior in, reset / posterior out)
    double* w_post;        // [M] posterior weights (before any reset)
    double* neff;          // [1]
    int32_t* resampled;    // [1]
    int32_t* status;       // [1] 1: every posterior weight was zero
    int32_t* idx;          // [M] resampled indices
    int32_t* src;          // [M] particle held by each slot afterwards
    int32_t* cnt;          // [M] scratch: duplicates per particle
    int32_t* copy_dst;     // [M] slots to overwrite
    int32_t* copy_src;     // [M] their sources
    int32_t* n_copy;       // [1]
    float* rain_mult;      // [M]
    float* scale;          // [M]
    MemberClock* ms;       // current member slot
    int M, G;
};

void launch_gauge(const float* state, const MemberClock* ms, const int32_t* cells, int G, int M,
                  int ld, int nx, size_t plane, float* y, cudaStream_t s);
void launch_pf(const PfArgs& a, cudaStream_t s);
void launch_copy(float* state, const MemberClock* ms, const int32_t* n_copy, const int32_t* dsts,
                 const int32_t* srcs, int M, size_t plane, int n_sm, cudaStream_t s);
void launch_resample(int M, const double* w, double u, int32_t* idx, cudaStream_t s);
int launch_storage(const float* state, const MemberClock* ms, int M, int ny, int nx, int ld,
                   size_t plane, double area, double* part, int part_cap, double* out,
                   cudaStream_t s);
void launch_hmax(const float* state, MemberClock* ms, int M, int ny, int nx, int ld, size_t plane,
                 int n_sm, cudaStream_t s);

}  // namespace flood
