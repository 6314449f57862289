// Internal: the grid handle behind the C ABI and host helpers shared by
// flood_capi.cu and adjoint_capi.cu.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "flood_internal.cuh"
#include "trace.cuh"

struct flood_grid {
    int ny = 0, nx = 0, ld = 0;
    size_t plane = 0;
    flood_params p{};
    float* zn = nullptr;          // [2][ny][ld]: z plane then n plane
    float* z = nullptr;           // = zn
    float* n = nullptr;           // = zn + plane
    int n_sm = 0;
    int engine = 1;               // 0: direct loads, 1: TMA-staged tiles
    long long wait_budget = -1;   // TMA row-wait limit of the step in clock cycles (< 0: default)
    CUtensorMap static_map{};
    CUtensorMap state_map{};
    CUtensorMap hm_map;          // running maxima, for the TMA step (tracking)
    CUtensorMap static_map_lc;   // land cover: the bed and each cell's class code (zc), the
                                 // TMA step's static planes (the roughness comes from the class)
    float* zc = nullptr;         // [2][ny][ld] land cover: bed, then class codes (uint32 bits)
    bool maps_ok = false;
    // ensemble
    int M = 0, nb = 0;
    float* state = nullptr;       // [2][M][3][plane]
    float* rain_mult = nullptr;   // [M]
    float* scale = nullptr;       // [M]
    float* hyeto = nullptr;       // [nb]
    double* w = nullptr;          // [M]
    double* w_post = nullptr;     // [M]
    flood::MemberClock* ms = nullptr;  // [3][M]
    double* vacc = nullptr;       // [M][nslot][2]
    int nslot = 0;
    double* rain_acc = nullptr;   // [M]
    int* err = nullptr;           // device error word
    int rows_per_strip = 64;
    int members_per_cta = 4;
    bool launch_fixed = false;    // set by flood_set_launch
    // particle filter
    int G = 0, G_cap = 0;
    int32_t* cells = nullptr;     // [G_cap]
    float* y = nullptr;           // [M][G_cap] last gauge sample
    float* y_in = nullptr;        // [M][G_cap] caller-supplied outputs
    double* d = nullptr;          // [G_cap]
    double* sigma = nullptr;      // [G_cap]
    float* beta = nullptr;        // [M]
    int32_t* pfi = nullptr;       // idx, src, cnt, copy_dst, copy_src: 5 x [M]
    int32_t* pf_small = nullptr;  // n_copy, resampled, status
    double* neff = nullptr;       // [1]
    double* part = nullptr;       // storage partials
    int part_cap = 0;
    double* storage = nullptr;    // [M]
    int64_t k = 0;                // step launches so far (member-slot rotation)
    int64_t launches = 0;         // all kernel launches
    // optional per-launch timing of the step kernel (CUDA events on the
    // launching stream)
    bool profile = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free;
    double prof_ms = 0.0;
    int64_t prof_launches = 0;
    // CUDA-graph replay of flood_step's launches (flood_set_graphs): a run of
    // kGraphSteps steps captured on cap_stream and replayed on the caller's
    // stream while the launch arguments stay those of graph_key
    bool graphs = false;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> graph_key;
    int64_t graph_launch_delta = 0;  // kernel launches of one replay
    int64_t graph_captures = 0, graph_replays = 0;
    // adjoint (flood_adjoint): step log, checkpoints, segment replay buffers
    flood::MemberPlan* plan = nullptr;  // [M] the current step's plans
    flood::MemberPlan* log = nullptr;   // [M][log_cap] plans of the logged steps
    int log_cap = 0;
    bool logging = false;         // step kernels record dt and checkpoints
    float* ckpt = nullptr;        // [n_ckpt][M][3][plane]
    size_t ckpt_floats = 0;
    int ckpt_every = 0;
    float* seg = nullptr;         // [slots][M][3][plane]
    size_t seg_floats = 0;
    float* lam = nullptr;         // [2][M][3][plane]
    float* gnm = nullptr;         // [M][plane] per-member Manning gradients
    float* gn_out = nullptr;      // [ny][nx]
    double* gpart = nullptr;      // [M][nslot][2]
    int* seg_end = nullptr;       // [M]
    int32_t* samp_step = nullptr; // [ns][M]
    float* samp_y = nullptr;      // [ns][M][G]
    double* samp_d = nullptr;     // [ns][G]
    int32_t* samp_cells = nullptr;
    double adj_fwd_ms = 0.0, adj_rev_ms = 0.0;
    // land cover (land_cover.cu; Section 4.1)
    bool lc_on = false;
    int lc_K = 0;
    uint8_t* cls8 = nullptr;      // [ny][ld] class of every cell
    uint8_t lc_out_mask = 0;      // bit q: class q lies outside the domain
    std::vector<uint8_t> lc_span_out;  // [ny][spans] 1: the row's 128-column span lies wholly
                                       // outside the domain
    int2* tiles = nullptr;        // [n_tiles] (span, strip) tiles holding a cell of the domain
    int n_tiles = 0, tiles_rows = 0;  // built for strips of tiles_rows rows (0: not built)
    float lc_n0[4] = {0, 0, 0, 0};       // class Manning n (the members' default)
    float lc_runoff[4] = {1, 1, 1, 1};   // fraction of the rain that stays
    float lc_drains[4] = {0, 0, 0, 0};   // 1: the member's drainage applies
    double lc_rain_cells = 0.0;   // sum over cells of the runoff fraction
    float* lc_n = nullptr;        // [M][4] per-member class roughness
    float* lc_drain = nullptr;    // [M] per-member drainage rate (m/s)
    double* dacc = nullptr;       // [M][nslot] drained volume partials
    float* lc_adj = nullptr;      // [M + 3][plane] the reverse pass's fields: the bed, each
                                  // member's Manning n, the share of the rain that stays,
                                  // the drainage flag
    double* gdpart = nullptr;     // [M][nslot] drainage-rate gradient partials
    std::vector<double> adj_gdrain;  // [M] dL/d(drainage rate) of the last adjoint
    double* lc_cgrad = nullptr;   // [M][4] per-class Manning gradients of the last adjoint
    double* lc_dgrad = nullptr;   // [M] drainage-rate gradients (device copy, calibration)
    // inflow hydrograph (inflow.cu)
    float* inflow = nullptr;      // [inflow_blocks] discharge per rain block (m^3/s)
    int inflow_blocks = 0, in_r0 = 0, in_r1 = 0;
    double* inflow_acc = nullptr; // [M] inflow volume
    // ensemble products (products.cu)
    float* hmax_field = nullptr;  // [M][plane] running maximum depth of each member
    long long* prod_u = nullptr;  // [384] the products' weights in units of 2^-60
    bool track_max = false;
    // gradient calibration (calibrate.cu)
    float* n0 = nullptr;          // [ny][ld] base roughness, kept once a factor field is set
    float* fac = nullptr;         // [fcy][fcx] roughness factor field
    double* fgrad = nullptr;      // [fcy][fcx] dL/df of the last adjoint
    double* closs = nullptr;      // [2][closs_cap] per-member losses and rain gradients
    int fcy = 0, fcx = 0, closs_cap = 0;
    uint64_t epoch = 0;           // bumped by every change of the ensemble or of its inputs
    uint64_t adj_epoch = ~0ull;   // epoch right after the last flood_adjoint
    bool adj_gn = false;          // that adjoint computed the Manning gradient
    int adj_ns = 0, adj_G = 0;    // its samples and gauges (samp_y, samp_d)
    int adj_nslot = 0;            // volume slots per member in its gpart
    std::string msg;
};


namespace flood {

int fail(flood_grid* g, int code, const std::string& m);
int dalloc_bytes(flood_grid* g, void** p, size_t bytes);
template <class T>
int dalloc(flood_grid* g, T** p, size_t count)
{
    return dalloc_bytes(g, reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}
StepArgs step_args(const flood_grid* g, double t_end);
int launch_steps(flood_grid* g, int64_t count, double t_end, cudaStream_t s);
int read_clocks(flood_grid* g, std::vector<MemberClock>& out, cudaStream_t s);
int check_err(flood_grid* g);
void collect_profile(flood_grid* g);
void launch_copy_planes(float* field, const int32_t* n_copy, const int32_t* dsts, const int32_t* srcs,
                        size_t plane, int n_sm, cudaStream_t s);
int land_ensemble_init(flood_grid* g);  // per-member land-cover defaults after flood_ensemble_init
// Fill g->lc_adj from the classes and the members' current class roughness.
int land_adjoint_fields(flood_grid* g, cudaStream_t s);
// The calibration step with land cover: one joint step per member over its
// rain multiplier and land-cover parameters (loss, rain_grad: [M] on the
// device, rain_grad = dL_i/d(rain multiplier of i)).
int land_calibration_step(flood_grid* g, const double* loss, const double* rain_grad, double eta,
                          double delta, cudaStream_t s);
// The (span, strip) tiles of the current strip height that hold a cell of
// the domain (land cover with cells outside it), rebuilt when the strip
// height changes.
int land_tiles(flood_grid* g);
// Cells outside the domain stay dry and at rest: zero their depth and link
// fluxes in both state buffers of members [m0, m0 + count).
void land_zero_outside(flood_grid* g, int m0, int count, cudaStream_t s);
void launch_land_permute(float* lc_n, float* lc_drain, const int32_t* src, const int32_t* resampled,
                         int M, cudaStream_t s);

}  // namespace flood

#define FLOOD_CK(g, call)                                                                    \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return flood::fail((g), e_ == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA, \
                               std::string(#call) + ": " + cudaGetErrorString(e_));          \
    } while (0)
