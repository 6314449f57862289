// Reverse-mode kernels of the step (adjoint_kernel.cu).
#pragma once

#include "flood_internal.cuh"

namespace flood {

struct AdjArgs {
    const float* seg;        // [slots][M][3][plane] forward states of the segment
    float* lam;              // [2][M][3][plane] sensitivities (h, qx, qy)
    int lam_in;              // buffer holding the sensitivities to the step's outputs
    float* gn;               // [M][plane] per-member dL/dn_base (or null)
    double* gpart;           // [M][nslot][2] per-warp partials of dL/d(rain mult), dL/d(scale)
    const float* z;
    const float* n;          // Manning n of member m at n + m * n_mstride
    size_t n_mstride;        // 0 (one field for all members) or plane (land cover)
    const float* rw;         // [ny][ld] fraction of the rain that stays (land cover), or null
    const float* dflag;      // [ny][ld] 1 where the member's drainage applies (land cover)
    // land cover, TMA form: the member's Manning n of every class [M][4] and
    // the classes' runoff shares and drainage flags (the cells' classes come
    // with the staged rows)
    const float* lc_n;
    float lc_runoff[4];
    float lc_drains[4];
    double* gdpart;          // [M][nslot] per-warp partials of dL/d(drainage rate) (land cover)
    const float* scale;      // [M]
    const MemberPlan* log;   // [M][dt_log_cap] plans of the recorded steps
    const int* seg_end;      // [M] first step index past this segment, per member
    int dt_log_cap;
    int seg_first;           // step index whose input state sits in slot 0
    int rev_i;               // this launch handles step seg_end[m] - 1 - rev_i of member m
    size_t plane;
    int ny, nx, ld, M, rows_per_strip, nslot;
    double g, dxd;
    float h_eps, edge_drop;
    int limiter, east_out, south_out;
    int* err;                // device error word (bit 1: a bounded wait gave up)
};

// Tensor maps of the TMA-staged adjoint (adjoint_tma.cu): 136-column boxes of
// one row.
struct AdjTmaArgs {
    CUtensorMap seg_map;     // seg as (ld, ny, slots * M * 3), box of 3 planes (h, qx, qy)
    CUtensorMap seg1_map;    // the same memory, box of 1 plane (the depth after a step)
    CUtensorMap lam_map;     // lam as (ld, ny, 2 * M * 3), box of 3 planes
    CUtensorMap static_map;  // z, n as (ld, ny, 2), box of 2 planes; land cover: z and the
                             // class codes (one uint32 per cell), the same layout
    CUtensorMap gn_map;      // per-member Manning gradients as (ld, ny, M), box of 1 plane
    AdjArgs a;
};

void launch_adjoint(const AdjArgs& a, int members_per_cta, cudaStream_t s);
void launch_adjoint_tma(const AdjTmaArgs& t, int members_per_cta, cudaStream_t s);
int adjoint_tma_box_cols();
void launch_seed(const AdjArgs& a, const int32_t* sample_step, const float* y, const double* d,
                 const int32_t* cells, int ns, int G, cudaStream_t s);
void launch_reduce_members(const float* gm, int M, int ny, int nx, int ld, size_t plane, float* out,
                           cudaStream_t s);

}  // namespace flood
