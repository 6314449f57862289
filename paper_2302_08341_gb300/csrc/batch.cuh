// Uneven batches: many independent scenarios, each with its own grid, bed,
// roughness, rain and duration, stepped by one launch per step (extension
// beyond the paper).
#pragma once

#include "flood_internal.cuh"

namespace flood {

struct ScenDesc {
    float* state;          // [2][3][plane] (two buffers of h, qx, qy)
    const float* z;        // [ny][ld]
    const float* n;        // [ny][ld]
    const float* hyeto;    // [nb] rain rate per block (m/s)
    size_t plane;
    int ny, nx, ld, nb;
    float rain_mult, scale;
    double t_end;          // the scenario's own end time
    double ncell;          // cells the rain falls on (with land cover: the sum of runoff shares)
    // land cover (Section 4.1; lc = 0: none): the scenario's class of every
    // cell and per-class runoff share and drainage flag, the member's
    // Manning n of every class and drainage rate
    const uint8_t* cls;    // [ny][ld]
    float lc_n[4];
    float lc_runoff[4];
    float lc_drains[4];
    float lc_drain;        // m/s
    int lc;
};

// The land-cover tables of a member for one step, as for the ensemble's
// members (land_k): lane q of every group of four holds class q's entries,
// read from the descriptor in global memory (indexed by lane, a copy in
// registers would move to local memory).
__device__ __forceinline__ LandK batch_land_k(const ScenDesc* sd, float dr, double dt, int lane)
{
    LandK lk;
    lk.cls = sd->cls;
    const int q = lane & 3;
    lk.n = sd->lc_n[q];
    lk.dr = __fmul_rn(dr, sd->lc_runoff[q]);
    lk.dd = __fmul_rn(__fmul_rn(sd->lc_drain, sd->lc_drains[q]), (float)dt);
    return lk;
}

// One warp's work: a 128-column span of rows [r0, r1) of one scenario.
struct WarpTask {
    int scen, c0, r0, r1;
    int slot;              // this task's FP64 volume slot
    int first;             // 1 for the task that owns the scenario's clock
};

struct BatchArgs {
    const ScenDesc* scen;
    const WarpTask* tasks;
    int ntasks;
    const MemberClock* ms_in;  // [S] slot k%3
    MemberClock* ms_out;       // slot (k+1)%3
    MemberClock* ms_clr;       // slot (k+2)%3
    const double* t_stop;      // window end (device scalar, so captured graphs are reusable)
    MemberPlan* plan;          // [S] this step's plans
    double* vacc;              // [nslot_total][2]
    double* dacc;              // [nslot_total] drained volume partials (land cover)
    int lc;                    // every scenario has land cover (0: none has)
    double* rain_acc;          // [S]
    int* err;
    double alpha_dx, g, dt_cap, dt_fixed, h_floor, rain_block, dxd, cell_area;
    float h_eps, edge_drop;
    int limiter, east_out, south_out;
    const CUtensorMap* maps;   // [S][2] per entry: state (ld, ny, 6 planes); z and n, or with
                               // land cover z and the class codes (ld, ny, 2)
};

// The persistent form: one cooperative launch loops plan phase -> grid
// barrier -> step phase (warps draw tasks from a counter) -> grid barrier
// until no scenario is active (or max_steps).  The barrier is a counter and
// a generation word with bounded spins: a wait that runs out sets bit 2 of
// the error word (FLOOD_ERR_TIMEOUT) and every CTA leaves at its next
// barrier.
struct PersistArgs {
    BatchArgs a;               // ms_in/ms_out/ms_clr unused: slots rotate with k
    MemberClock* ms;           // [3][S]
    int S;
    int max_steps;
    int64_t k0;                // the batch's step counter when launched
    unsigned* bar;             // [2] arrivals, generation
    unsigned* task_next;       // [2] next task of the step phase, by step parity
    int* any_active;           // [2] some scenario steps, by step parity
    int64_t* steps_done;       // steps the launch advanced the clocks by
    long long budget;          // clock cycles a barrier wait may take
    int* diag;                 // [8] where the first wait gave up (kind, step, CTA, ...)
};

void launch_batch_plan(const BatchArgs& a, int n_scen, cudaStream_t s);
cudaError_t launch_batch_persistent(const PersistArgs& q, cudaStream_t s);
void launch_batch_step(const BatchArgs& a, int warps_per_cta, cudaStream_t s);
void launch_batch_step_tma(const BatchArgs& a, int warps_per_cta, cudaStream_t s);
int batch_tma_prepare();  // shared-memory attributes; call before any stream capture

}  // namespace flood
