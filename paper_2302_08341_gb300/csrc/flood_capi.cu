// Host side of the C ABI declared in include/flood.h: argument checks,
// device buffers, the step driver (per-member clocks, landing on t_end) and
// the particle-filter sequence.  Every step of the method runs in the
// kernels of step_kernel.cu and pf_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "grid.cuh"
#include "pf_kernels.cuh"
#include "tma.cuh"

using flood::MemberClock;

namespace {
thread_local std::string g_static_msg;
}  // namespace

namespace flood {

int fail(flood_grid* g, int code, const std::string& m)
{
    if (g) g->msg = m; else g_static_msg = m;
    return code;
}

int dalloc_bytes(flood_grid* g, void** p, size_t bytes)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess)
        return fail(g, e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return FLOOD_OK;
}

}  // namespace flood

using flood::fail;
using flood::dalloc;

namespace {

#define CK(g, call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((g), e_ == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

void dfree(void* p)
{
    if (p) cudaFree(p);
}

void free_ensemble(flood_grid* g)
{
    dfree(g->state); dfree(g->rain_mult); dfree(g->scale); dfree(g->hyeto); dfree(g->w);
    dfree(g->w_post); dfree(g->ms); dfree(g->vacc); dfree(g->rain_acc); dfree(g->y);
    dfree(g->y_in); dfree(g->beta); dfree(g->pfi); dfree(g->pf_small); dfree(g->neff);
    dfree(g->part); dfree(g->storage); dfree(g->cells); dfree(g->d); dfree(g->sigma);
    dfree(g->plan); dfree(g->log); dfree(g->ckpt); dfree(g->seg); dfree(g->lam);
    dfree(g->gnm); dfree(g->gn_out); dfree(g->gpart); dfree(g->seg_end); dfree(g->samp_step);
    dfree(g->samp_y); dfree(g->samp_d); dfree(g->samp_cells); dfree(g->closs);
    dfree(g->hmax_field); dfree(g->lc_n); dfree(g->lc_drain); dfree(g->dacc);
    dfree(g->inflow_acc); dfree(g->lc_adj); dfree(g->lc_cgrad); dfree(g->gdpart); dfree(g->lc_dgrad);
    g->inflow_acc = nullptr; g->lc_adj = nullptr; g->lc_cgrad = nullptr; g->gdpart = nullptr;
    g->lc_dgrad = nullptr;
    g->adj_gdrain.clear();
    g->closs = nullptr; g->closs_cap = 0; g->hmax_field = nullptr; g->track_max = false;
    g->lc_n = nullptr; g->lc_drain = nullptr; g->dacc = nullptr;
    g->plan = nullptr; g->log = nullptr; g->ckpt = nullptr; g->seg = nullptr;
    g->lam = nullptr; g->gnm = nullptr; g->gn_out = nullptr; g->gpart = nullptr;
    g->seg_end = nullptr; g->samp_step = nullptr; g->samp_y = nullptr; g->samp_d = nullptr;
    g->samp_cells = nullptr; g->log_cap = 0; g->ckpt_floats = 0; g->seg_floats = 0;
    g->logging = false;
    g->state = nullptr; g->rain_mult = nullptr; g->scale = nullptr; g->hyeto = nullptr;
    g->w = nullptr; g->w_post = nullptr; g->ms = nullptr; g->vacc = nullptr;
    g->rain_acc = nullptr; g->y = nullptr; g->y_in = nullptr; g->beta = nullptr;
    g->pfi = nullptr; g->pf_small = nullptr; g->neff = nullptr; g->part = nullptr;
    g->storage = nullptr; g->cells = nullptr; g->d = nullptr; g->sigma = nullptr;
    g->M = 0; g->G = 0; g->G_cap = 0;
}

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace flood {

StepArgs step_args(const flood_grid* g, double t_end)
{
    flood::StepArgs a{};
    a.state = g->state;
    a.z = g->z;
    a.n = g->n;
    a.rain_mult = g->rain_mult;
    a.scale = g->scale;
    a.hyeto = g->hyeto;
    const int64_t k = g->k;
    a.ms_in = g->ms + (k % 3) * g->M;
    a.ms_out = g->ms + ((k + 1) % 3) * g->M;
    a.ms_clr = g->ms + ((k + 2) % 3) * g->M;
    a.vacc = g->vacc;
    a.rain_acc = g->rain_acc;
    a.plan = g->plan;
    a.log = g->logging ? g->log : nullptr;
    a.dt_log_cap = g->log_cap;
    a.ckpt = g->logging ? g->ckpt : nullptr;
    a.ckpt_every = g->ckpt_every > 0 ? g->ckpt_every : 1;
    a.err = g->err;
    a.wait_budget = g->wait_budget < 0 ? flood::kTmaWaitBudgetDefault : g->wait_budget;
    a.hmax_field = g->track_max ? g->hmax_field : nullptr;
    a.lc_on = g->lc_on ? 1 : 0;
    if (g->lc_on) {
        a.cls = g->cls8;
        a.lc_n = g->lc_n;
        a.lc_drain = g->lc_drain;
        for (int q = 0; q < 4; ++q) {
            a.lc_runoff[q] = g->lc_runoff[q];
            a.lc_drains[q] = g->lc_drains[q];
        }
        a.dacc = g->dacc;
    }
    a.plane = g->plane;
    a.ny = g->ny; a.nx = g->nx; a.ld = g->ld; a.M = g->M; a.nb = g->nb;
    a.rows_per_strip = g->rows_per_strip;
    a.nslot = g->nslot;
    a.t_end = t_end;
    a.alpha_dx = g->p.alpha * g->p.dx;
    a.g = g->p.g;
    a.dt_cap = g->p.dt_cap;
    a.dt_fixed = g->p.dt_fixed;
    a.h_floor = g->p.h_floor;
    a.rain_block = g->p.rain_block;
    a.dxd = g->p.dx;
    a.cell_area = g->p.dx * g->p.dx;
    a.ncell = g->lc_on ? g->lc_rain_cells : (double)g->ny * (double)g->nx;
    if (g->inflow && g->inflow_acc) {
        a.inflow = g->inflow;
        a.inflow_blocks = g->inflow_blocks;
        a.in_r0 = g->in_r0;
        a.in_r1 = g->in_r1;
        a.inflow_acc = g->inflow_acc;
    }
    a.dx = (float)g->p.dx;
    a.h_eps = (float)g->p.h_eps;
    a.edge_drop = (float)(g->p.edge_slope * g->p.dx);
    a.limiter = g->p.limiter;
    a.east_out = g->p.east_outflow;
    a.south_out = g->p.south_outflow;
    return a;
}

// Fold finished timing pairs into the totals (after a synchronisation).
void collect_profile(flood_grid* g)
{
    for (auto& p : g->ev_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) {
            g->prof_ms += ms;
            g->prof_launches++;
        }
        g->ev_free.push_back(p);
    }
    g->ev_pending.clear();
}

// Whether the TMA step leaves out the tiles wholly outside the domain (land
// cover with classes outside it; the ordinary step only).
static bool skips_tiles(const flood_grid* g, const StepArgs& a)
{
    return g->engine == 1 && g->maps_ok && a.lc_on && g->lc_out_mask && !a.ckpt &&
           a.wait_budget == kTmaWaitBudgetDefault;
}

// One step of every member: the plan kernel (Eq. 4, the events), then the
// step kernel of the chosen engine.
static int launch_one(flood_grid* g, double t_end, cudaStream_t s)
{
    flood::StepArgs a = step_args(g, t_end);
    flood::launch_plan(a, s);
    g->launches++;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (g->profile) {
        if (g->ev_free.empty()) {
            CK(g, cudaEventCreate(&ev.first));
            CK(g, cudaEventCreate(&ev.second));
        } else {
            ev = g->ev_free.back();
            g->ev_free.pop_back();
        }
        CK(g, cudaEventRecord(ev.first, s));
    }
    if (g->engine == 1 && g->maps_ok) {
        flood::TmaArgs t;
        t.state_map = g->state_map;
        t.static_map = a.lc_on ? g->static_map_lc : g->static_map;
        if (a.hmax_field) t.hm_map = g->hm_map;
        if (skips_tiles(g, a)) {
            if (g->tiles_rows != g->rows_per_strip) {
                const int rc = land_tiles(g);
                if (rc) return rc;
            }
            a.tiles = g->tiles;
            a.n_tiles = g->n_tiles;
        }
        t.a = a;
        if (flood::launch_step_tma(t, g->members_per_cta, s))
            return fail(g, FLOOD_ERR_STATE, "a changed wait budget covers the plain step only");
    } else if (g->engine == 2 && !g->lc_on) {
        flood::launch_step_per_member(a, s);
        g->launches += g->M - 1;
    } else {
        flood::launch_step(a, g->members_per_cta, s);
    }
    if (g->profile) {
        CK(g, cudaEventRecord(ev.second, s));
        g->ev_pending.push_back(ev);
    }
    g->k++;
    g->launches++;
    return FLOOD_OK;
}

// Steps per captured run: a multiple of the member-clock ring's period (3),
// so that a run captured at ring phase 0 replays at every later phase 0.
static constexpr int kGraphSteps = 24;

// Everything the launches of a step take from the host, at ring phase 0: the
// step arguments (t_end included), the engine and its launch shape, the
// tensor maps and the tile list.  A captured run replays while this holds.
static std::vector<unsigned char> graph_key(const flood_grid* g, double t_end)
{
    const flood::StepArgs a = step_args(g, t_end);
    std::vector<unsigned char> key;
    auto put = [&key](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        key.insert(key.end(), b, b + n);
    };
    put(&a, sizeof a);
    const int v[4] = {g->engine, g->members_per_cta, g->maps_ok ? 1 : 0, g->n_tiles};
    put(v, sizeof v);
    put(&g->tiles, sizeof g->tiles);
    if (g->engine == 1 && g->maps_ok) {
        put(&g->state_map, sizeof g->state_map);
        put(a.lc_on ? &g->static_map_lc : &g->static_map, sizeof(CUtensorMap));
        if (a.hmax_field) put(&g->hm_map, sizeof g->hm_map);
    }
    return key;
}

// Capture kGraphSteps steps from ring phase 0 on the grid's own stream
// (nothing runs; the steps' kernels become the graph's nodes in order),
// unless the graph in hand was captured from the same launch arguments.
static int ensure_graph(flood_grid* g, double t_end)
{
    CK(g, cudaGetLastError());  // the plain launches before this one
    if (skips_tiles(g, step_args(g, t_end)) && g->tiles_rows != g->rows_per_strip) {
        const int rc = land_tiles(g);  // allocates: not while capturing
        if (rc) return rc;
    }
    std::vector<unsigned char> key = graph_key(g, t_end);
    if (g->gexec && key == g->graph_key) return FLOOD_OK;
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->gexec = nullptr;
    g->graph = nullptr;
    g->graph_key.clear();
    if (!g->cap_stream) CK(g, cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    const int64_t k0 = g->k, l0 = g->launches;
    CK(g, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed));
    int rc = FLOOD_OK;
    for (int i = 0; i < kGraphSteps && rc == FLOOD_OK; ++i) rc = launch_one(g, t_end, g->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(g->cap_stream, &graph);
    g->graph_launch_delta = g->launches - l0;
    g->k = k0;
    g->launches = l0;
    cudaGetLastError();  // a failed capture is reported below, not by the next check
    if (rc != FLOOD_OK || ec != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return rc != FLOOD_OK ? rc
                              : fail(g, FLOOD_ERR_CUDA,
                                     std::string("capturing the steps: ") + cudaGetErrorString(ec));
    }
    const cudaError_t ei = cudaGraphInstantiate(&g->gexec, graph, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        g->gexec = nullptr;
        return fail(g, FLOOD_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
    }
    g->graph = graph;
    g->graph_key = std::move(key);
    g->graph_captures++;
    return FLOOD_OK;
}

int launch_steps(flood_grid* g, int64_t count, double t_end, cudaStream_t s)
{
    g->epoch++;
    int64_t i = 0;
    // runs of kGraphSteps steps from a captured graph (steps timed one by one
    // and the adjoint's logged steps launch plainly); the steps before ring
    // phase 0 and the remainder launch plainly
    if (g->graphs && !g->profile && !g->logging && count >= kGraphSteps + 2) {
        for (; g->k % 3 != 0; ++i) {
            const int rc = launch_one(g, t_end, s);
            if (rc) return rc;
        }
        const int rc = ensure_graph(g, t_end);
        if (rc) return rc;
        for (; count - i >= kGraphSteps; i += kGraphSteps) {
            CK(g, cudaGraphLaunch(g->gexec, s));
            g->k += kGraphSteps;
            g->launches += g->graph_launch_delta;
            g->graph_replays++;
        }
    }
    for (; i < count; ++i) {
        const int rc = launch_one(g, t_end, s);
        if (rc) return rc;
    }
    CK(g, cudaGetLastError());
    return FLOOD_OK;
}

int check_err(flood_grid* g)
{
    int err = 0;
    CK(g, cudaMemcpy(&err, g->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 2) return fail(g, FLOOD_ERR_TIMEOUT, "a bounded wait for staged tiles gave up");
    if (err) return fail(g, FLOOD_ERR_NAN, "a kernel produced a non-finite depth");
    return FLOOD_OK;
}

int read_clocks(flood_grid* g, std::vector<MemberClock>& out, cudaStream_t s)
{
    out.resize(g->M);
    CK(g, cudaMemcpyAsync(out.data(), g->ms + (g->k % 3) * g->M, sizeof(MemberClock) * g->M,
                          cudaMemcpyDeviceToHost, s));
    CK(g, cudaStreamSynchronize(s));
    collect_profile(g);
    return check_err(g);
}

// Grow the per-warp volume slots when a launch shape with more warp tasks
// per member is chosen; the sums accumulated so far move to slot 0.
int ensure_vacc(flood_grid* g, int need)
{
    if (!g->M || need <= g->nslot) return FLOOD_OK;
    const int M = g->M;
    std::vector<double> old((size_t)M * g->nslot * 2), nw((size_t)M * need * 2, 0.0);
    CK(g, cudaDeviceSynchronize());
    CK(g, cudaMemcpy(old.data(), g->vacc, sizeof(double) * old.size(), cudaMemcpyDeviceToHost));
    for (int m = 0; m < M; ++m)
        for (int k = 0; k < g->nslot; ++k)
            for (int j = 0; j < 2; ++j)
                nw[(size_t)m * need * 2 + j] += old[((size_t)m * g->nslot + k) * 2 + j];
    int rc = dalloc(g, &g->vacc, nw.size());
    if (rc) return rc;
    CK(g, cudaMemcpy(g->vacc, nw.data(), sizeof(double) * nw.size(), cudaMemcpyHostToDevice));
    if (g->dacc) {  // drained volume (land cover): the same folding
        std::vector<double> od((size_t)M * g->nslot), nd((size_t)M * need, 0.0);
        CK(g, cudaMemcpy(od.data(), g->dacc, sizeof(double) * od.size(), cudaMemcpyDeviceToHost));
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < g->nslot; ++k) nd[(size_t)m * need] += od[(size_t)m * g->nslot + k];
        if ((rc = dalloc(g, &g->dacc, nd.size()))) return rc;
        CK(g, cudaMemcpy(g->dacc, nd.data(), sizeof(double) * nd.size(), cudaMemcpyHostToDevice));
    }
    g->nslot = need;
    return FLOOD_OK;
}

}  // namespace flood

using flood::launch_steps;
using flood::read_clocks;
using flood::collect_profile;
using flood::ensure_vacc;

namespace {

int choose_rows_per_strip(int ny, int nx, int M, int n_sm)
{
    const int spans = (nx + 127) / 128;
    int rh = 64;
    while (rh > 4 && (int64_t)M * spans * ((ny + rh - 1) / rh) < (int64_t)n_sm * 32) rh /= 2;
    return rh;
}

}  // namespace

extern "C" {

void flood_default_params(flood_params* p)
{
    if (!p) return;
    p->dx = 3.0;
    p->g = 9.81;
    p->alpha = 0.7;
    p->dt_cap = 1.0;
    p->dt_fixed = 0.0;
    p->h_eps = 0.0;
    p->h_floor = 1e-6;
    p->rain_block = 300.0;
    p->edge_slope = 0.005;
    p->limiter = 1;
    p->east_outflow = 1;
    p->south_outflow = 0;
    p->reserved = 0;
}

const char* flood_last_error(const flood_grid* g)
{
    return g ? g->msg.c_str() : g_static_msg.c_str();
}

int flood_create_grid(flood_grid** out, int ny, int nx, const float* z, const float* n_base,
                      const flood_params* p)
{
    if (!out) return fail(nullptr, FLOOD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ny < 1 || nx < 1) return fail(nullptr, FLOOD_ERR_ARG, "ny and nx must be >= 1");
    if ((int64_t)ny * nx > (int64_t)1 << 31) return fail(nullptr, FLOOD_ERR_ARG, "grid too large");
    if (!z || !n_base || !p) return fail(nullptr, FLOOD_ERR_ARG, "z, n_base and p are required");
    if (!(p->dx > 0) || !(p->g > 0) || !(p->dt_cap > 0) || !(p->rain_block > 0) ||
        !(p->alpha > 0) || p->dt_fixed < 0 || p->h_eps < 0 || p->reserved != 0)
        return fail(nullptr, FLOOD_ERR_ARG, "invalid flood_params");
    flood_grid* g = new flood_grid();
    g->ny = ny;
    g->nx = nx;
    g->ld = (nx + 31) / 32 * 32;
    g->plane = (size_t)ny * g->ld;
    g->p = *p;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (g->n_sm <= 0) g->n_sm = 1;
    int rc;
    if ((rc = dalloc(g, &g->zn, 2 * g->plane)) || (rc = dalloc(g, &g->err, 1))) {
        g_static_msg = g->msg;
        flood_destroy(g);
        return rc;
    }
    g->z = g->zn;
    g->n = g->zn + g->plane;
    cudaError_t e = cudaMemset(g->zn, 0, sizeof(float) * 2 * g->plane);
    if (e == cudaSuccess) e = cudaMemset(g->err, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy2D(g->z, sizeof(float) * g->ld, z, sizeof(float) * nx, sizeof(float) * nx, ny,
                         cudaMemcpyDefault);
    if (e == cudaSuccess)
        e = cudaMemcpy2D(g->n, sizeof(float) * g->ld, n_base, sizeof(float) * nx,
                         sizeof(float) * nx, ny, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        fail(nullptr, FLOOD_ERR_CUDA, std::string("flood_create_grid: ") + cudaGetErrorString(e));
        flood_destroy(g);
        return FLOOD_ERR_CUDA;
    }
    if (flood::encode_map_3d(&g->static_map, g->zn, g->ld, g->ny, 2, sizeof(float) * g->ld,
                             sizeof(float) * g->plane, flood::tma_box_cols(), 1, 2) != 0)
        g->engine = 0;  // no tensor-map encoder: direct loads only
    *out = g;
    return FLOOD_OK;
}

int flood_destroy(flood_grid* g)
{
    if (!g) return FLOOD_OK;
    cudaDeviceSynchronize();
    collect_profile(g);
    for (auto& p : g->ev_free) {
        cudaEventDestroy(p.first);
        cudaEventDestroy(p.second);
    }
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    free_ensemble(g);
    dfree(g->zn);
    dfree(g->err);
    dfree(g->n0); dfree(g->fac); dfree(g->fgrad);
    dfree(g->inflow);
    dfree(g->tiles);
    dfree(g->prod_u);
    dfree(g->zc);
    delete g;
    return FLOOD_OK;
}

int flood_ensemble_init(flood_grid* g, int M, const float* h0, int h0_per_member,
                        const float* rain_mult, const float* manning_scale,
                        const float* hyetograph, int n_blocks, double t0, void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (M < 1) return fail(g, FLOOD_ERR_ARG, "n_members must be >= 1");
    if (!rain_mult || !manning_scale) return fail(g, FLOOD_ERR_ARG, "rain_mult and manning_scale are required");
    if (n_blocks < 0 || (n_blocks > 0 && !hyetograph)) return fail(g, FLOOD_ERR_ARG, "bad hyetograph");
    if (!(t0 >= 0.0)) return fail(g, FLOOD_ERR_ARG, "t0 must be >= 0");
    cudaStream_t s = S(stream);
    CK(g, cudaStreamSynchronize(s));
    g->epoch++;
    free_ensemble(g);
    g->M = M;
    g->nb = n_blocks;
    if (!g->launch_fixed) {
        g->rows_per_strip = choose_rows_per_strip(g->ny, g->nx, M, g->n_sm);
        g->members_per_cta = M >= 4 ? 4 : 1;
    }
    g->nslot = flood::step_nslot(g->ny, g->nx, g->rows_per_strip);
    g->part_cap = (g->ny + 15) / 16;
    int rc;
    if ((rc = dalloc(g, &g->state, (size_t)2 * M * 3 * g->plane)) ||
        (rc = dalloc(g, &g->rain_mult, M)) || (rc = dalloc(g, &g->scale, M)) ||
        (rc = dalloc(g, &g->hyeto, n_blocks)) || (rc = dalloc(g, &g->w, M)) ||
        (rc = dalloc(g, &g->w_post, M)) || (rc = dalloc(g, &g->ms, (size_t)3 * M)) ||
        (rc = dalloc(g, &g->vacc, (size_t)M * g->nslot * 2)) || (rc = dalloc(g, &g->rain_acc, M)) ||
        (rc = dalloc(g, &g->inflow_acc, M)) ||
        (rc = dalloc(g, &g->beta, M)) || (rc = dalloc(g, &g->pfi, (size_t)5 * M)) ||
        (rc = dalloc(g, &g->pf_small, 4)) || (rc = dalloc(g, &g->neff, 1)) ||
        (rc = dalloc(g, &g->part, (size_t)M * g->part_cap)) || (rc = dalloc(g, &g->storage, M)) ||
        (rc = dalloc(g, &g->plan, M))) {
        free_ensemble(g);
        return rc;
    }
    CK(g, cudaMemsetAsync(g->state, 0, sizeof(float) * 2 * (size_t)M * 3 * g->plane, s));
    g->maps_ok = flood::encode_map_3d(&g->state_map, g->state, g->ld, g->ny, (uint64_t)2 * M * 3,
                                      sizeof(float) * g->ld, sizeof(float) * g->plane,
                                      flood::tma_box_cols(), 1, 3) == 0;
    if (h0) {
        for (int m = 0; m < M; ++m) {
            const float* src = h0 + (h0_per_member ? (size_t)m * g->ny * g->nx : 0);
            CK(g, cudaMemcpy2DAsync(g->state + (size_t)m * 3 * g->plane, sizeof(float) * g->ld, src,
                                    sizeof(float) * g->nx, sizeof(float) * g->nx, g->ny,
                                    cudaMemcpyDefault, s));
        }
    }
    CK(g, cudaMemcpyAsync(g->rain_mult, rain_mult, sizeof(float) * M, cudaMemcpyDefault, s));
    CK(g, cudaMemcpyAsync(g->scale, manning_scale, sizeof(float) * M, cudaMemcpyDefault, s));
    if (n_blocks > 0)
        CK(g, cudaMemcpyAsync(g->hyeto, hyetograph, sizeof(float) * n_blocks, cudaMemcpyDefault, s));
    std::vector<double> w(M, 1.0 / M);
    CK(g, cudaMemcpyAsync(g->w, w.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
    std::vector<MemberClock> ms((size_t)3 * M);
    for (auto& c : ms) { c.t = t0; c.steps = 0; c.hmax_bits = 0; c.cur = 0; }
    CK(g, cudaMemcpyAsync(g->ms, ms.data(), sizeof(MemberClock) * 3 * M, cudaMemcpyHostToDevice, s));
    CK(g, cudaMemsetAsync(g->vacc, 0, sizeof(double) * M * g->nslot * 2, s));
    CK(g, cudaMemsetAsync(g->rain_acc, 0, sizeof(double) * M, s));
    CK(g, cudaMemsetAsync(g->inflow_acc, 0, sizeof(double) * M, s));
    CK(g, cudaMemsetAsync(g->err, 0, sizeof(int), s));
    g->k = 0;
    flood::launch_hmax(g->state, g->ms, M, g->ny, g->nx, g->ld, g->plane, g->n_sm, s);
    g->launches++;
    CK(g, cudaGetLastError());
    CK(g, cudaStreamSynchronize(s));
    if (g->lc_on && (rc = flood::land_ensemble_init(g))) return rc;
    return FLOOD_OK;
}

int flood_step(flood_grid* g, int n_steps, double t_end, void* stream)
{
    const flood::TraceRange range("flood_step");
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    cudaStream_t s = S(stream);
    if (t_end < 0.0) {
        if (n_steps < 0) return fail(g, FLOOD_ERR_ARG, "n_steps must be >= 0");
        return launch_steps(g, n_steps, -1.0, s);
    }
    int64_t done = 0;
    std::vector<MemberClock> c;
    double last_tmin = -1.0;
    for (int rounds = 0;; ++rounds) {
        int rc = read_clocks(g, c, s);
        if (rc) return rc;
        double tmin = t_end;
        for (int m = 0; m < g->M; ++m) tmin = std::min(tmin, c[m].t);
        if (rounds > 0 && tmin < t_end && !(tmin > last_tmin))
            return fail(g, FLOOD_ERR_STATE, "members stopped advancing toward t_end");
        last_tmin = tmin;
        int64_t need = 0;
        for (int m = 0; m < g->M; ++m) {
            if (c[m].t >= t_end) continue;
            double dt;
            if (g->p.dt_fixed > 0) {
                dt = g->p.dt_fixed;
            } else {
                float hf;
                std::memcpy(&hf, &c[m].hmax_bits, sizeof(hf));
                double hm = std::max((double)hf, g->p.h_floor);
                dt = std::min(g->p.alpha * g->p.dx / std::sqrt(g->p.g * hm), g->p.dt_cap);
            }
            const double rb = g->p.rain_block;
            const int64_t edges = (int64_t)std::floor(t_end / rb) - (int64_t)std::floor(c[m].t / rb) + 1;
            need = std::max(need, (int64_t)std::ceil((t_end - c[m].t) / dt) + edges);
        }
        if (need == 0) break;
        if (need > (int64_t)1 << 26)
            return fail(g, FLOOD_ERR_STATE, "reaching t_end would take more than 2^26 steps");
        if (n_steps > 0) need = std::min<int64_t>(need, n_steps - done);
        if (need <= 0) break;
        if ((rc = launch_steps(g, need, t_end, s))) return rc;
        done += need;
    }
    return FLOOD_OK;
}

int flood_gauge_sample(flood_grid* g, int G, const int32_t* cell_idx, float* y_out, void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (G < 1 || !cell_idx) return fail(g, FLOOD_ERR_ARG, "need n_gauges >= 1 and cell_idx");
    cudaStream_t s = S(stream);
    std::vector<int32_t> cells(G);
    CK(g, cudaMemcpy(cells.data(), cell_idx, sizeof(int32_t) * G, cudaMemcpyDefault));
    for (int k = 0; k < G; ++k)
        if (cells[k] < 0 || (int64_t)cells[k] >= (int64_t)g->ny * g->nx)
            return fail(g, FLOOD_ERR_ARG, "gauge cell index out of range");
    if (G > g->G_cap) {
        int rc;
        if ((rc = dalloc(g, &g->cells, G)) || (rc = dalloc(g, &g->y, (size_t)g->M * G)) ||
            (rc = dalloc(g, &g->y_in, (size_t)g->M * G)) || (rc = dalloc(g, &g->d, G)) ||
            (rc = dalloc(g, &g->sigma, G)))
            return rc;
        g->G_cap = G;
    }
    g->G = G;
    CK(g, cudaMemcpyAsync(g->cells, cells.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, s));
    flood::launch_gauge(g->state, g->ms + (g->k % 3) * g->M, g->cells, G, g->M, g->ld, g->nx,
                        g->plane, g->y, s);
    g->launches++;
    CK(g, cudaGetLastError());
    if (y_out)
        CK(g, cudaMemcpyAsync(y_out, g->y, sizeof(float) * g->M * G, cudaMemcpyDefault, s));
    return FLOOD_OK;
}

int pf_assimilate(flood_grid* g, int G, const float* y, const double* d, const double* sigma,
                  double sigma_rel, double n_thr_frac, int force_resample, double u,
                  const float* beta, double* weights_out, int32_t* idx_out, double* neff_out,
                  int32_t* resampled_out, void* stream)
{
    const flood::TraceRange range("pf_assimilate");
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (G < 1 || !d || (!sigma && !(sigma_rel > 0)) || !beta)
        return fail(g, FLOOD_ERR_ARG, "need n_gauges >= 1, d, sigma (or sigma_rel) and beta");
    if (!(u >= 0.0 && u < 1.0)) return fail(g, FLOOD_ERR_ARG, "u must lie in [0, 1)");
    cudaStream_t s = S(stream);
    g->epoch++;
    if (!y && G != g->G)
        return fail(g, FLOOD_ERR_STATE, "y is NULL but no gauge sample of this size exists");
    if (G > g->G_cap) {
        int rc;
        if ((rc = dalloc(g, &g->y, (size_t)g->M * G)) ||
            (rc = dalloc(g, &g->y_in, (size_t)g->M * G)) || (rc = dalloc(g, &g->d, G)) ||
            (rc = dalloc(g, &g->sigma, G)) || (rc = dalloc(g, &g->cells, G)))
            return rc;
        g->G_cap = G;
        g->G = 0;
    }
    const float* ydev = g->y;
    if (y) {
        CK(g, cudaMemcpyAsync(g->y_in, y, sizeof(float) * g->M * G, cudaMemcpyDefault, s));
        ydev = g->y_in;
    }
    CK(g, cudaMemcpyAsync(g->d, d, sizeof(double) * G, cudaMemcpyDefault, s));
    if (sigma) CK(g, cudaMemcpyAsync(g->sigma, sigma, sizeof(double) * G, cudaMemcpyDefault, s));
    CK(g, cudaMemcpyAsync(g->beta, beta, sizeof(float) * g->M, cudaMemcpyDefault, s));
    const int M = g->M;
    flood::PfArgs a{};
    a.y = ydev;
    a.d = g->d;
    a.sigma = g->sigma;
    a.sigma_rel = sigma_rel;
    a.n_thr_frac = n_thr_frac;
    a.force = force_resample;
    a.u = u;
    a.beta = g->beta;
    a.w = g->w;
    a.w_post = g->w_post;
    a.neff = g->neff;
    a.n_copy = g->pf_small;
    a.resampled = g->pf_small + 1;
    a.status = g->pf_small + 2;
    a.idx = g->pfi;
    a.src = g->pfi + M;
    a.cnt = g->pfi + 2 * M;
    a.copy_dst = g->pfi + 3 * M;
    a.copy_src = g->pfi + 4 * M;
    a.rain_mult = g->rain_mult;
    a.scale = g->scale;
    a.ms = g->ms + (g->k % 3) * M;
    a.M = M;
    a.G = G;
    flood::launch_pf(a, s);
    flood::launch_copy(g->state, a.ms, a.n_copy, a.copy_dst, a.copy_src, M, g->plane, g->n_sm, s);
    g->launches += 2;
    if (g->lc_on) {  // land-cover parameters follow their particle
        flood::launch_land_permute(g->lc_n, g->lc_drain, a.src, a.resampled, M, s);
        g->launches++;
    }
    if (g->track_max) {
        flood::launch_copy_planes(g->hmax_field, a.n_copy, a.copy_dst, a.copy_src, g->plane, g->n_sm, s);
        g->launches++;
    }
    CK(g, cudaGetLastError());
    if (weights_out) CK(g, cudaMemcpyAsync(weights_out, g->w_post, sizeof(double) * M, cudaMemcpyDefault, s));
    if (idx_out) CK(g, cudaMemcpyAsync(idx_out, a.idx, sizeof(int32_t) * M, cudaMemcpyDefault, s));
    if (neff_out) CK(g, cudaMemcpyAsync(neff_out, g->neff, sizeof(double), cudaMemcpyDefault, s));
    if (resampled_out)
        CK(g, cudaMemcpyAsync(resampled_out, a.resampled, sizeof(int32_t), cudaMemcpyDefault, s));
    return FLOOD_OK;
}

int pf_resample_systematic(int n, const double* w, double u, int32_t* idx, void* stream)
{
    if (n < 1 || !w || !idx) return fail(nullptr, FLOOD_ERR_ARG, "need n >= 1, w and idx");
    if (!(u >= 0.0 && u < 1.0)) return fail(nullptr, FLOOD_ERR_ARG, "u must lie in [0, 1)");
    cudaStream_t s = S(stream);
    double* dw = nullptr;
    int32_t* di = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dw, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&di, sizeof(int32_t) * n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w, sizeof(double) * n, cudaMemcpyDefault, s);
    if (e == cudaSuccess) {
        flood::launch_resample(n, dw, u, di, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx, di, sizeof(int32_t) * n, cudaMemcpyDefault, s);
    if (dw) cudaFreeAsync(dw, s);
    if (di) cudaFreeAsync(di, s);
    if (e != cudaSuccess)
        return fail(nullptr, FLOOD_ERR_CUDA, std::string("pf_resample_systematic: ") + cudaGetErrorString(e));
    return FLOOD_OK;
}

int flood_get_state(flood_grid* g, int member, float* h, float* qx, float* qy, void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (member < 0 || member >= g->M) return fail(g, FLOOD_ERR_ARG, "member out of range");
    cudaStream_t s = S(stream);
    MemberClock c;
    CK(g, cudaMemcpyAsync(&c, g->ms + (g->k % 3) * g->M + member, sizeof(c), cudaMemcpyDeviceToHost, s));
    CK(g, cudaStreamSynchronize(s));
    const float* base = g->state + (size_t)(c.cur * g->M + member) * 3 * g->plane;
    float* outs[3] = {h, qx, qy};
    for (int k = 0; k < 3; ++k)
        if (outs[k])
            CK(g, cudaMemcpy2DAsync(outs[k], sizeof(float) * g->nx, base + k * g->plane,
                                    sizeof(float) * g->ld, sizeof(float) * g->nx, g->ny,
                                    cudaMemcpyDefault, s));
    return FLOOD_OK;
}

int flood_set_state(flood_grid* g, int member, const float* h, const float* qx, const float* qy,
                    void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (member < 0 || member >= g->M) return fail(g, FLOOD_ERR_ARG, "member out of range");
    cudaStream_t s = S(stream);
    g->epoch++;
    MemberClock* slot = g->ms + (g->k % 3) * g->M + member;
    MemberClock c;
    CK(g, cudaMemcpyAsync(&c, slot, sizeof(c), cudaMemcpyDeviceToHost, s));
    CK(g, cudaStreamSynchronize(s));
    float* base = g->state + (size_t)(c.cur * g->M + member) * 3 * g->plane;
    const float* ins[3] = {h, qx, qy};
    for (int k = 0; k < 3; ++k)
        if (ins[k])
            CK(g, cudaMemcpy2DAsync(base + k * g->plane, sizeof(float) * g->ld, ins[k],
                                    sizeof(float) * g->nx, sizeof(float) * g->nx, g->ny,
                                    cudaMemcpyDefault, s));
    // cells outside the domain stay dry and at rest whatever was given for them
    if (g->lc_on) flood::land_zero_outside(g, member, 1, s);
    if (h) {  // refresh the member's maximum depth (input of Eq. 4)
        CK(g, cudaMemsetAsync(&slot->hmax_bits, 0, sizeof(uint32_t), s));
        flood::launch_hmax(g->state, g->ms + (g->k % 3) * g->M, g->M, g->ny, g->nx, g->ld, g->plane,
                           g->n_sm, s);
        g->launches++;
    }
    CK(g, cudaGetLastError());
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}

int flood_get_members(flood_grid* g, double* t, int64_t* steps, float* rain_mult,
                      float* manning_scale, double* weights, float* hmax)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    const int M = g->M;
    CK(g, cudaDeviceSynchronize());
    std::vector<MemberClock> c(M);
    CK(g, cudaMemcpy(c.data(), g->ms + (g->k % 3) * M, sizeof(MemberClock) * M, cudaMemcpyDeviceToHost));
    for (int m = 0; m < M; ++m) {
        if (t) t[m] = c[m].t;
        if (steps) steps[m] = c[m].steps;
        if (hmax) std::memcpy(&hmax[m], &c[m].hmax_bits, sizeof(float));
    }
    if (rain_mult) CK(g, cudaMemcpy(rain_mult, g->rain_mult, sizeof(float) * M, cudaMemcpyDefault));
    if (manning_scale) CK(g, cudaMemcpy(manning_scale, g->scale, sizeof(float) * M, cudaMemcpyDefault));
    if (weights) CK(g, cudaMemcpy(weights, g->w, sizeof(double) * M, cudaMemcpyDefault));
    return FLOOD_OK;
}

int flood_set_members(flood_grid* g, const float* rain_mult, const float* manning_scale,
                      const double* weights)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    const int M = g->M;
    g->epoch++;
    CK(g, cudaDeviceSynchronize());
    if (rain_mult) CK(g, cudaMemcpy(g->rain_mult, rain_mult, sizeof(float) * M, cudaMemcpyDefault));
    if (manning_scale) CK(g, cudaMemcpy(g->scale, manning_scale, sizeof(float) * M, cudaMemcpyDefault));
    if (weights) CK(g, cudaMemcpy(g->w, weights, sizeof(double) * M, cudaMemcpyDefault));
    return FLOOD_OK;
}

int flood_volume_report(flood_grid* g, double* storage, double* rain, double* outflow,
                        double* clamp)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    const int M = g->M;
    CK(g, cudaDeviceSynchronize());
    if (storage) {
        if (flood::launch_storage(g->state, g->ms + (g->k % 3) * M, M, g->ny, g->nx, g->ld, g->plane,
                                  g->p.dx * g->p.dx, g->part, g->part_cap, g->storage, 0))
            return fail(g, FLOOD_ERR_STATE, "storage partial buffer too small");
        g->launches += 2;
        CK(g, cudaGetLastError());
        CK(g, cudaMemcpy(storage, g->storage, sizeof(double) * M, cudaMemcpyDefault));
    }
    if (rain) CK(g, cudaMemcpy(rain, g->rain_acc, sizeof(double) * M, cudaMemcpyDefault));
    if (outflow || clamp) {
        std::vector<double> v((size_t)M * g->nslot * 2);
        CK(g, cudaMemcpy(v.data(), g->vacc, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
        for (int m = 0; m < M; ++m) {
            double o = 0.0, c = 0.0;
            for (int k = 0; k < g->nslot; ++k) {
                o += v[((size_t)m * g->nslot + k) * 2];
                c += v[((size_t)m * g->nslot + k) * 2 + 1];
            }
            if (outflow) outflow[m] = o;
            if (clamp) clamp[m] = c;
        }
    }
    return FLOOD_OK;
}

int64_t flood_launch_count(const flood_grid* g) { return g ? g->launches : 0; }

int flood_profile(flood_grid* g, int enable, double* step_kernel_ms, int64_t* step_launches)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    CK(g, cudaDeviceSynchronize());
    collect_profile(g);
    if (step_kernel_ms) *step_kernel_ms = g->prof_ms;
    if (step_launches) *step_launches = g->prof_launches;
    g->prof_ms = 0.0;
    g->prof_launches = 0;
    g->profile = enable != 0;
    return FLOOD_OK;
}

int flood_set_launch(flood_grid* g, int rows_per_strip, int members_per_cta)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (rows_per_strip == 0 && members_per_cta == 0) {
        g->launch_fixed = false;
        if (g->M) {
            const int rh = choose_rows_per_strip(g->ny, g->nx, g->M, g->n_sm);
            int rc = ensure_vacc(g, flood::step_nslot(g->ny, g->nx, rh));
            if (rc) return rc;
            g->rows_per_strip = rh;
            g->members_per_cta = g->M >= 4 ? 4 : 1;
        }
        return FLOOD_OK;
    }
    if (rows_per_strip < 1 || rows_per_strip > 4096)
        return fail(g, FLOOD_ERR_ARG, "rows_per_strip must lie in [1, 4096]");
    if (members_per_cta != 1 && members_per_cta != 2 && members_per_cta != 4 && members_per_cta != 8)
        return fail(g, FLOOD_ERR_ARG, "members_per_cta must be 1, 2, 4 or 8");
    int rc = ensure_vacc(g, flood::step_nslot(g->ny, g->nx, rows_per_strip));
    if (rc) return rc;
    g->rows_per_strip = rows_per_strip;
    g->members_per_cta = members_per_cta;
    g->launch_fixed = true;
    return FLOOD_OK;
}

int flood_set_engine(flood_grid* g, int engine)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (engine < 0 || engine > 2) return fail(g, FLOOD_ERR_ARG, "engine must be 0, 1 or 2");
    g->engine = engine;
    return FLOOD_OK;
}

int flood_set_wait_budget(flood_grid* g, int64_t cycles)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    g->wait_budget = cycles < 0 ? -1 : (long long)cycles;
    return FLOOD_OK;
}

int flood_set_graphs(flood_grid* g, int on)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    g->graphs = on != 0;
    return FLOOD_OK;
}

int flood_graph_stats(flood_grid* g, int64_t* captures, int64_t* replays)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (captures) *captures = g->graph_captures;
    if (replays) *replays = g->graph_replays;
    return FLOOD_OK;
}

int flood_get_launch(const flood_grid* g, int* rows_per_strip, int* members_per_cta)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (rows_per_strip) *rows_per_strip = g->rows_per_strip;
    if (members_per_cta) *members_per_cta = g->members_per_cta;
    return FLOOD_OK;
}

int flood_sync(flood_grid* g, void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    CK(g, cudaStreamSynchronize(S(stream)));
    return flood::check_err(g);
}

}  // extern "C"

// ---- autotuner ------------------------------------------------------------
// Times candidate step-kernel configurations (engine x rows per strip x
// members per CTA) on the live ensemble and keeps the fastest.  The ensemble
// is snapshotted first (current state, clocks, volume counters) and restored
// afterwards, so tuning leaves the simulation untouched.
extern "C" int flood_autotune(flood_grid* g, int steps_per_trial, int* best_rows, int* best_mpc,
                              int* best_engine, double* best_ms, void* stream)
{
    if (!g) return fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (steps_per_trial < 1) steps_per_trial = 4;
    steps_per_trial = (steps_per_trial + 2) / 3 * 3;  // whole clock-slot cycles
    cudaStream_t s = S(stream);
    const int M = g->M;
    const size_t ms = 3 * g->plane;
    std::vector<MemberClock> c0;
    int rc = read_clocks(g, c0, s);
    if (rc) return rc;
    float* snap = nullptr;
    if ((rc = dalloc(g, &snap, (size_t)M * ms))) return rc;
    for (int m = 0; m < M; ++m)
        CK(g, cudaMemcpyAsync(snap + (size_t)m * ms, g->state + (size_t)(c0[m].cur * M + m) * ms,
                              sizeof(float) * ms, cudaMemcpyDeviceToDevice, s));
    std::vector<double> rain0(M), vacc0((size_t)M * g->nslot * 2), drained0(M, 0.0);
    CK(g, cudaMemcpy(rain0.data(), g->rain_acc, sizeof(double) * M, cudaMemcpyDeviceToHost));
    CK(g, cudaMemcpy(vacc0.data(), g->vacc, sizeof(double) * vacc0.size(), cudaMemcpyDeviceToHost));
    std::vector<double> inflow0(M);
    CK(g, cudaMemcpy(inflow0.data(), g->inflow_acc, sizeof(double) * M, cudaMemcpyDeviceToHost));
    if (g->dacc) {
        std::vector<double> d0((size_t)M * g->nslot);
        CK(g, cudaMemcpy(d0.data(), g->dacc, sizeof(double) * d0.size(), cudaMemcpyDeviceToHost));
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < g->nslot; ++k) drained0[m] += d0[(size_t)m * g->nslot + k];
    }
    const int64_t k0 = g->k;
    const int rows0 = g->rows_per_strip, mpc0 = g->members_per_cta, eng0 = g->engine;
    const bool fixed0 = g->launch_fixed;
    const bool track0 = g->track_max;  // trial steps must not raise the running maxima
    g->track_max = false;
    struct Cand { int rows, mpc, engine; };
    std::vector<Cand> cands;
    // members per CTA: the TMA engine's plain step also has 2 and 8 (the
    // land-cover and tracking forms run 2 as 1 and 8 as 4, so those are not
    // timed twice)
    const bool plain_tma = !g->lc_on && !g->track_max;
    for (int e : {1, 0})
        for (int r : {32, 64, 128})
            for (int mp : {8, 4, 2, 1}) {
                if (e == 1 && !g->maps_ok) continue;
                if ((mp == 2 || mp == 8) && !(e == 1 && plain_tma)) continue;
                if (mp > M) continue;
                cands.push_back({r, mp, e});
            }
    cudaEvent_t e0, e1;
    CK(g, cudaEventCreate(&e0));
    CK(g, cudaEventCreate(&e1));
    double best = 1e300;
    Cand bc{rows0, mpc0, eng0};
    for (const Cand& cd : cands) {
        if ((rc = flood_set_launch(g, cd.rows, cd.mpc))) break;
        g->engine = cd.engine;
        if ((rc = launch_steps(g, 3, -1.0, s))) break;  // warm-up
        CK(g, cudaEventRecord(e0, s));
        if ((rc = launch_steps(g, steps_per_trial, -1.0, s))) break;
        CK(g, cudaEventRecord(e1, s));
        CK(g, cudaEventSynchronize(e1));
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        const double per = t / steps_per_trial;
        if (per < best) {
            best = per;
            bc = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore the ensemble exactly as it was
    std::vector<MemberClock> cn;
    int rc2 = read_clocks(g, cn, s);
    if (!rc2) {
        for (int m = 0; m < M; ++m)
            cudaMemcpyAsync(g->state + (size_t)(cn[m].cur * M + m) * ms, snap + (size_t)m * ms,
                            sizeof(float) * ms, cudaMemcpyDeviceToDevice, s);
        std::vector<MemberClock> back = c0;
        for (int m = 0; m < M; ++m) back[m].cur = cn[m].cur;
        cudaMemcpyAsync(g->ms + (g->k % 3) * M, back.data(), sizeof(MemberClock) * M,
                        cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(g->rain_acc, rain0.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(g->inflow_acc, inflow0.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s);
    }
    cudaStreamSynchronize(s);
    cudaFree(snap);
    g->track_max = track0;
    (void)k0;
    if (rc) {
        g->rows_per_strip = rows0;
        g->members_per_cta = mpc0;
        g->engine = eng0;
        g->launch_fixed = fixed0;
        return rc;
    }
    if (rc2) return rc2;
    if ((rc = flood_set_launch(g, bc.rows, bc.mpc))) return rc;
    g->engine = bc.engine;
    // volume slots now follow the chosen shape; restore the saved sums into slot 0 of each member
    {
        std::vector<double> v((size_t)M * g->nslot * 2, 0.0);
        for (int m = 0; m < M; ++m)
            for (size_t kk = 0; kk < vacc0.size() / M / 2; ++kk)
                for (int j = 0; j < 2; ++j)
                    v[(size_t)m * g->nslot * 2 + j] += vacc0[((size_t)m * (vacc0.size() / M / 2) + kk) * 2 + j];
        CK(g, cudaMemcpy(g->vacc, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
        if (g->dacc) {
            std::vector<double> d((size_t)M * g->nslot, 0.0);
            for (int m = 0; m < M; ++m) d[(size_t)m * g->nslot] = drained0[m];
            CK(g, cudaMemcpy(g->dacc, d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice));
        }
    }
    if (best_rows) *best_rows = bc.rows;
    if (best_mpc) *best_mpc = bc.mpc;
    if (best_engine) *best_engine = bc.engine;
    if (best_ms) *best_ms = best;
    return FLOOD_OK;
}
