// Host side of the uneven-batch API (flood_batch_*): per-scenario buffers,
// the flat warp-task table, and the step driver that replays a CUDA graph of
// kGraphSteps step launches until every scenario has reached the window end.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/flood.h"
#include "batch.cuh"
#include "trace.cuh"
#include "pf_kernels.cuh"
#include "tma.cuh"

using flood::MemberClock;

namespace {

constexpr int kGraphSteps = 96;  // a multiple of 3: clock slots line up across replays
constexpr int kSpan = 128;

thread_local std::string g_batch_msg;

}  // namespace

// A batch holds n_scen scenarios (grid, bed, roughness, storm, end time) and
// S entries: the members of every scenario, scenario by scenario, each with
// its own state, clock, rain multiplier and Manning scale.  Everything the
// step kernels index (descriptors, clocks, plans, tensor maps, tasks) is per
// entry; the members of a scenario share its bed, roughness and storm.
struct flood_batch {
    int S = 0;                        // entries (members of all scenarios)
    int n_scen = 0;
    flood_params p{};
    std::vector<int> ny, nx, ld;      // per entry (the scenario's)
    std::vector<int> sny, snx, sld;   // per scenario
    std::vector<int> scen_of;         // [S] the scenario of each entry
    std::vector<int> first;           // [n_scen + 1] first entry of each scenario
    std::vector<float*> zn, hyeto;    // per scenario
    std::vector<float*> state;        // per entry: [2][3][plane]
    std::vector<flood::ScenDesc> desc;
    flood::ScenDesc* d_desc = nullptr;
    std::vector<flood::WarpTask> tasks;
    flood::WarpTask* d_tasks = nullptr;
    std::vector<int> slot0;           // first volume slot of each scenario
    int nslot = 0;
    MemberClock* ms = nullptr;        // [3][S]
    double* vacc = nullptr;           // [nslot][2]
    double* rain_acc = nullptr;       // [S]
    double* storage = nullptr;        // [S]
    double* part = nullptr;           // storage partials
    int part_cap = 0;
    int* err = nullptr;
    double* t_stop = nullptr;         // device scalar
    flood::MemberPlan* plan = nullptr; // [S]
    int rows_per_strip = 64, warps_per_cta = 4;
    int engine = 0;                   // 0: direct loads, 1: TMA-staged rows, 2: persistent
    unsigned* pbar = nullptr;         // persistent form: barrier words [2], task counters [2]
    int* pact = nullptr;              // [2] some scenario steps, by step parity
    int64_t* pdone = nullptr;         // steps the last persistent launch advanced the clocks by
    int* pdiag = nullptr;             // [8] where a persistent launch's first wait gave up
    long long wait_budget = -1;       // grid-barrier wait limit in clock cycles (< 0: default)
    CUtensorMap* d_maps = nullptr;    // [S][2] tensor maps of each entry
    bool tma_ok = false;              // the tensor-map encoder is available
    bool initialised = false;
    int64_t k = 0, launches = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    // land cover per scenario (Section 4.1), set before flood_batch_init for
    // every scenario or for none
    std::vector<int> lc;                        // 1: the scenario has land cover
    std::vector<uint8_t*> cls8;                 // class of every cell [ny][ld]
    std::vector<float*> zc;                     // bed and class codes [2][ny][ld] (TMA engines)
    std::vector<int> lc_K;                      // classes
    std::vector<std::array<float, 4>> lc_runoff, lc_drains, lc_n0;
    std::vector<double> lc_rain_cells;          // sum of the runoff shares over the cells
    std::vector<std::vector<uint8_t>> span_out; // [ny][spans]: 1 where a row's span lies outside
    double* dacc = nullptr;                     // [nslot] drained volume partials
    bool lc_all = false;                        // every scenario has land cover
    std::string msg;
};

namespace {

int bfail(flood_batch* b, int code, const std::string& m)
{
    if (b) b->msg = m; else g_batch_msg = m;
    return code;
}

#define BCK(b, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

cudaStream_t S_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void drop_graph(flood_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Task table: for each scenario, strips of rows_per_strip rows x 128-column
// spans in row-major order (neighbouring warps share halo rows in L2), and
// for each tile the scenario's members one after another, so that the warps
// taking one tile for different members are neighbours and the tile's bed
// and roughness come from DRAM once for all of them (Section 3.2's shared
// definitive data, as in the ensemble kernel).
int build_tasks(flood_batch* b)
{
    b->tasks.clear();
    b->slot0.assign(b->S, 0);
    std::vector<std::vector<int>> slots(b->S);
    for (int sc = 0; sc < b->n_scen; ++sc) {
        const int e0 = b->first[sc], e1 = b->first[sc + 1];
        const int spans = (b->nx[e0] + kSpan - 1) / kSpan;
        const bool skip = b->lc[sc] && !b->span_out[sc].empty();
        for (int r0 = 0; r0 < b->ny[e0]; r0 += b->rows_per_strip)
            for (int sp = 0; sp < spans; ++sp) {
                // land cover: a tile wholly outside the domain stays dry and
                // at rest, so it is not scheduled (the same results)
                if (skip) {
                    bool out = true;
                    const int r1 = std::min(r0 + b->rows_per_strip, b->ny[e0]);
                    for (int r = r0; out && r < r1; ++r) out = b->span_out[sc][(size_t)r * spans + sp] != 0;
                    if (out) continue;
                }
                for (int e = e0; e < e1; ++e) {
                    flood::WarpTask t;
                    t.scen = e;
                    t.c0 = sp * kSpan;
                    t.r0 = r0;
                    t.r1 = std::min(r0 + b->rows_per_strip, b->ny[e]);
                    t.slot = 0;
                    t.first = (r0 == 0 && sp == 0) ? 1 : 0;
                    slots[e].push_back((int)b->tasks.size());
                    b->tasks.push_back(t);
                }
            }
    }
    // volume slots: each entry's tasks own consecutive slots
    int slot = 0;
    for (int e = 0; e < b->S; ++e) {
        b->slot0[e] = slots[e].empty() ? -1 : slot;  // -1: no tile of the entry is scheduled
        for (int ti : slots[e]) b->tasks[ti].slot = slot++;
    }
    if (b->d_tasks) cudaFree(b->d_tasks);
    b->d_tasks = nullptr;
    BCK(b, cudaMalloc(&b->d_tasks, sizeof(flood::WarpTask) * b->tasks.size()));
    BCK(b, cudaMemcpy(b->d_tasks, b->tasks.data(), sizeof(flood::WarpTask) * b->tasks.size(),
                      cudaMemcpyHostToDevice));
    // one FP64 volume slot per task (flood_batch_set_launch carries sums over)
    std::vector<double> nw((size_t)slot * 2, 0.0);
    if (b->vacc) cudaFree(b->vacc);
    b->vacc = nullptr;
    BCK(b, cudaMalloc(&b->vacc, sizeof(double) * nw.size()));
    BCK(b, cudaMemcpy(b->vacc, nw.data(), sizeof(double) * nw.size(), cudaMemcpyHostToDevice));
    if (b->dacc) cudaFree(b->dacc);
    b->dacc = nullptr;
    BCK(b, cudaMalloc(&b->dacc, sizeof(double) * std::max(slot, 1)));
    BCK(b, cudaMemset(b->dacc, 0, sizeof(double) * std::max(slot, 1)));
    b->nslot = slot;
    drop_graph(b);
    return FLOOD_OK;
}

flood::BatchArgs batch_args(const flood_batch* b, int64_t k)
{
    flood::BatchArgs a{};
    a.scen = b->d_desc;
    a.tasks = b->d_tasks;
    a.ntasks = (int)b->tasks.size();
    a.ms_in = b->ms + (k % 3) * b->S;
    a.ms_out = b->ms + ((k + 1) % 3) * b->S;
    a.ms_clr = b->ms + ((k + 2) % 3) * b->S;
    a.t_stop = b->t_stop;
    a.plan = b->plan;
    a.vacc = b->vacc;
    a.rain_acc = b->rain_acc;
    a.err = b->err;
    a.alpha_dx = b->p.alpha * b->p.dx;
    a.g = b->p.g;
    a.dt_cap = b->p.dt_cap;
    a.dt_fixed = b->p.dt_fixed;
    a.h_floor = b->p.h_floor;
    a.rain_block = b->p.rain_block;
    a.dxd = b->p.dx;
    a.cell_area = b->p.dx * b->p.dx;
    a.h_eps = (float)b->p.h_eps;
    a.edge_drop = (float)(b->p.edge_slope * b->p.dx);
    a.limiter = b->p.limiter;
    a.east_out = b->p.east_outflow;
    a.south_out = b->p.south_outflow;
    a.maps = b->d_maps;
    a.dacc = b->dacc;
    a.lc = b->lc_all ? 1 : 0;
    return a;
}

int ensure_graph(flood_batch* b)
{
    if (b->graph) return FLOOD_OK;
    if (!b->cap_stream) BCK(b, cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t gr;
    BCK(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < kGraphSteps; ++i) {
        const flood::BatchArgs a = batch_args(b, i);
        flood::launch_batch_plan(a, b->S, b->cap_stream);
        if (b->engine == 1)
            flood::launch_batch_step_tma(a, b->warps_per_cta, b->cap_stream);
        else
            flood::launch_batch_step(a, b->warps_per_cta, b->cap_stream);
    }
    BCK(b, cudaStreamEndCapture(b->cap_stream, &gr));
    cudaError_t e = cudaGraphInstantiate(&b->graph, gr, 0);
    cudaGraphDestroy(gr);
    BCK(b, e);
    return FLOOD_OK;
}

int read_batch_clocks(flood_batch* b, std::vector<MemberClock>& c, cudaStream_t s)
{
    c.resize(b->S);
    BCK(b, cudaMemcpyAsync(c.data(), b->ms + (b->k % 3) * b->S, sizeof(MemberClock) * b->S,
                           cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    int err = 0;
    BCK(b, cudaMemcpy(&err, b->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 2) return bfail(b, FLOOD_ERR_TIMEOUT, "a bounded device wait gave up");
    if (err) return bfail(b, FLOOD_ERR_NAN, "a kernel produced a non-finite depth");
    return FLOOD_OK;
}

// (Re)build the entries for counts[sc] members of every scenario: each
// entry's state (zeroed), descriptor, tensor maps, clocks, plans and sums,
// and the task table.  Frees the previous entries' buffers.
int set_entries(flood_batch* b, const std::vector<int>& counts)
{
    for (float* p : b->state)
        if (p) cudaFree(p);
    b->state.clear();
    void* old[] = {b->d_desc, b->ms, b->rain_acc, b->storage, b->plan, b->d_maps};
    for (void* p : old)
        if (p) cudaFree(p);
    b->d_desc = nullptr; b->ms = nullptr; b->rain_acc = nullptr; b->storage = nullptr;
    b->plan = nullptr; b->d_maps = nullptr;
    drop_graph(b);
    int S = 0;
    b->first.assign(b->n_scen + 1, 0);
    for (int sc = 0; sc < b->n_scen; ++sc) {
        b->first[sc] = S;
        S += counts[sc];
    }
    b->first[b->n_scen] = S;
    b->S = S;
    b->scen_of.assign(S, 0);
    b->ny.assign(S, 0); b->nx.assign(S, 0); b->ld.assign(S, 0);
    b->state.assign(S, nullptr);
    b->desc.assign(S, flood::ScenDesc{});
    for (int sc = 0; sc < b->n_scen; ++sc)
        for (int e = b->first[sc]; e < b->first[sc + 1]; ++e) {
            b->scen_of[e] = sc;
            b->ny[e] = b->sny[sc]; b->nx[e] = b->snx[sc]; b->ld[e] = b->sld[sc];
            const size_t plane = (size_t)b->sny[sc] * b->sld[sc];
            BCK(b, cudaMalloc(&b->state[e], sizeof(float) * 6 * plane));
            BCK(b, cudaMemset(b->state[e], 0, sizeof(float) * 6 * plane));
            flood::ScenDesc& d = b->desc[e];
            d.state = b->state[e];
            d.z = b->zn[sc];
            d.n = b->zn[sc] + plane;
            d.hyeto = b->hyeto[sc];
            d.plane = plane;
            d.ny = b->sny[sc];
            d.nx = b->snx[sc];
            d.ld = b->sld[sc];
            d.nb = 0;
            d.rain_mult = 1.0f;
            d.scale = 1.0f;
            d.t_end = 0.0;
            d.ncell = b->lc[sc] ? b->lc_rain_cells[sc] : (double)b->sny[sc] * b->snx[sc];
            d.lc = b->lc[sc];
            d.cls = b->lc[sc] ? b->cls8[sc] : nullptr;
            for (int q = 0; q < 4; ++q) {
                d.lc_n[q] = b->lc[sc] ? b->lc_n0[sc][q] : 0.0f;
                d.lc_runoff[q] = b->lc[sc] ? b->lc_runoff[sc][q] : 1.0f;
                d.lc_drains[q] = b->lc[sc] ? b->lc_drains[sc][q] : 0.0f;
            }
            d.lc_drain = 0.0f;
        }
    BCK(b, cudaMalloc(&b->ms, sizeof(MemberClock) * 3 * S));
    BCK(b, cudaMemset(b->ms, 0, sizeof(MemberClock) * 3 * S));
    BCK(b, cudaMalloc(&b->rain_acc, sizeof(double) * S));
    BCK(b, cudaMemset(b->rain_acc, 0, sizeof(double) * S));
    BCK(b, cudaMalloc(&b->storage, sizeof(double) * S));
    BCK(b, cudaMalloc(&b->plan, sizeof(flood::MemberPlan) * S));
    BCK(b, cudaMalloc(&b->d_desc, sizeof(flood::ScenDesc) * S));
    BCK(b, cudaMemcpy(b->d_desc, b->desc.data(), sizeof(flood::ScenDesc) * S, cudaMemcpyHostToDevice));
    // tensor maps of every entry for the TMA-staged step (direct loads if the
    // encoder is unavailable): its own state, its scenario's bed and
    // roughness (with land cover: the bed and the class codes)
    std::vector<CUtensorMap> maps((size_t)2 * S);
    bool ok = b->tma_ok;
    for (int e = 0; ok && e < S; ++e) {
        const int sc = b->scen_of[e];
        const uint64_t s1 = sizeof(float) * b->ld[e], s2 = sizeof(float) * b->desc[e].plane;
        ok = flood::encode_map_3d(&maps[2 * e], b->state[e], b->ld[e], b->ny[e], 6, s1, s2,
                                  flood::tma_box_cols(), 1, 3) == 0 &&
             flood::encode_map_3d(&maps[2 * e + 1], b->lc[sc] ? b->zc[sc] : b->zn[sc], b->ld[e],
                                  b->ny[e], 2, s1, s2, flood::tma_box_cols(), 1, 2) == 0;
    }
    if (ok) {
        BCK(b, cudaMalloc(&b->d_maps, sizeof(CUtensorMap) * maps.size()));
        BCK(b, cudaMemcpy(b->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                          cudaMemcpyHostToDevice));
    } else if (b->engine != 0) {
        b->engine = 0;
    }
    return build_tasks(b);
}

// Each entry's volume sums (outflow, clamp; drained) into the first slot of
// its tasks, the other slots zeroed (after the task table changed).
int put_entry_sums(flood_batch* b, const std::vector<double>& per, const std::vector<double>& dper)
{
    std::vector<double> v((size_t)b->nslot * 2, 0.0), dv(std::max(b->nslot, 1), 0.0);
    for (int i = 0; i < b->S; ++i) {
        if (b->slot0[i] < 0) continue;  // no task: nothing was summed
        v[(size_t)b->slot0[i] * 2] = per[(size_t)i * 2];
        v[(size_t)b->slot0[i] * 2 + 1] = per[(size_t)i * 2 + 1];
        dv[b->slot0[i]] = dper[i];
    }
    BCK(b, cudaMemcpy(b->vacc, v.data(), sizeof(double) * v.size(), cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->dacc, dv.data(), sizeof(double) * dv.size(), cudaMemcpyHostToDevice));
    return FLOOD_OK;
}

}  // namespace

extern "C" {

const char* flood_batch_last_error(const flood_batch* b)
{
    return b ? b->msg.c_str() : g_batch_msg.c_str();
}

int flood_batch_create(flood_batch** out, int n, const int32_t* ny, const int32_t* nx,
                       const float* const* z, const float* const* n_base, const flood_params* p)
{
    if (!out) return bfail(nullptr, FLOOD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !ny || !nx || !z || !n_base || !p)
        return bfail(nullptr, FLOOD_ERR_ARG, "need n >= 1 and every array");
    if (!(p->dx > 0) || !(p->g > 0) || !(p->dt_cap > 0) || !(p->rain_block > 0) || !(p->alpha > 0) ||
        p->dt_fixed < 0 || p->h_eps < 0 || p->reserved != 0)
        return bfail(nullptr, FLOOD_ERR_ARG, "invalid flood_params");
    for (int i = 0; i < n; ++i)
        if (ny[i] < 1 || nx[i] < 1 || !z[i] || !n_base[i])
            return bfail(nullptr, FLOOD_ERR_ARG, "scenario with an empty grid or missing field");
    flood_batch* b = new flood_batch();
    b->n_scen = n;
    b->p = *p;
    b->sny.assign(ny, ny + n);
    b->snx.assign(nx, nx + n);
    b->sld.resize(n);
    b->zn.assign(n, nullptr);
    b->hyeto.assign(n, nullptr);
    b->lc.assign(n, 0);
    b->cls8.assign(n, nullptr);
    b->zc.assign(n, nullptr);
    b->lc_K.assign(n, 0);
    b->lc_runoff.assign(n, {1.0f, 1.0f, 1.0f, 1.0f});
    b->lc_drains.assign(n, {0.0f, 0.0f, 0.0f, 0.0f});
    b->lc_n0.assign(n, {0.05f, 0.05f, 0.05f, 0.05f});
    b->lc_rain_cells.assign(n, 0.0);
    b->span_out.assign(n, {});
    auto bad = [&](cudaError_t e) {
        g_batch_msg = std::string("flood_batch_create: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? FLOOD_ERR_OOM : FLOOD_ERR_CUDA;
    };
    for (int i = 0; i < n; ++i) {
        b->sld[i] = (nx[i] + 31) / 32 * 32;
        const size_t plane = (size_t)ny[i] * b->sld[i];
        cudaError_t e = cudaMalloc(&b->zn[i], sizeof(float) * 2 * plane);
        if (e == cudaSuccess) e = cudaMemset(b->zn[i], 0, sizeof(float) * 2 * plane);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(b->zn[i], sizeof(float) * b->sld[i], z[i], sizeof(float) * nx[i],
                             sizeof(float) * nx[i], ny[i], cudaMemcpyDefault);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(b->zn[i] + plane, sizeof(float) * b->sld[i], n_base[i], sizeof(float) * nx[i],
                             sizeof(float) * nx[i], ny[i], cudaMemcpyDefault);
        if (e != cudaSuccess) {
            int rc = bad(e);
            flood_batch_destroy(b);
            return rc;
        }
    }
    cudaError_t e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->t_stop, sizeof(double));
    int maxny = *std::max_element(b->sny.begin(), b->sny.end());
    b->part_cap = (maxny + 15) / 16;
    if (e == cudaSuccess) e = cudaMalloc(&b->part, sizeof(double) * b->part_cap);
    if (e != cudaSuccess) {
        int rc = bad(e);
        flood_batch_destroy(b);
        return rc;
    }
    b->tma_ok = flood::batch_tma_prepare() == 0;
    b->engine = b->tma_ok ? 1 : 0;
    int rc = set_entries(b, std::vector<int>(n, 1));  // one member per scenario until init
    if (rc) {
        g_batch_msg = b->msg;
        flood_batch_destroy(b);
        return rc;
    }
    *out = b;
    return FLOOD_OK;
}

int flood_batch_destroy(flood_batch* b)
{
    if (!b) return FLOOD_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (float* p : b->zn) if (p) cudaFree(p);
    for (float* p : b->state) if (p) cudaFree(p);
    for (float* p : b->hyeto) if (p) cudaFree(p);
    for (float* p : b->zc) if (p) cudaFree(p);
    for (uint8_t* p : b->cls8) if (p) cudaFree(p);
    void* bufs[] = {b->d_desc, b->d_tasks, b->ms, b->vacc, b->rain_acc, b->storage, b->part,
                    b->err, b->t_stop, b->plan, b->d_maps, b->pbar, b->pact, b->pdone, b->pdiag,
                    b->dacc};
    for (void* p : bufs) if (p) cudaFree(p);
    delete b;
    return FLOOD_OK;
}

int flood_batch_init_members(flood_batch* b, const float* const* hyetographs,
                             const int32_t* n_blocks, const int32_t* n_members,
                             const float* rain_mult, const float* manning_scale,
                             const double* t_end, void* stream)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (!hyetographs || !n_blocks || !n_members || !rain_mult || !manning_scale || !t_end)
        return bfail(b, FLOOD_ERR_ARG, "every array is required");
    cudaStream_t s = S_(stream);
    BCK(b, cudaStreamSynchronize(s));
    std::vector<int> counts(b->n_scen);
    int64_t total = 0;
    for (int i = 0; i < b->n_scen; ++i) {
        if (n_members[i] < 1 || n_members[i] > 4096)
            return bfail(b, FLOOD_ERR_ARG, "every scenario needs 1..4096 members");
        if (n_blocks[i] < 0 || (n_blocks[i] > 0 && !hyetographs[i]) || !(t_end[i] >= 0.0))
            return bfail(b, FLOOD_ERR_ARG, "bad hyetograph or end time");
        counts[i] = n_members[i];
        total += n_members[i];
    }
    if (total > (1 << 20)) return bfail(b, FLOOD_ERR_ARG, "more than 2^20 members in all");
    const int n_lc = (int)std::count(b->lc.begin(), b->lc.end(), 1);
    if (n_lc != 0 && n_lc != b->n_scen)
        return bfail(b, FLOOD_ERR_STATE, "land cover must be set for every scenario or for none");
    b->lc_all = n_lc == b->n_scen;
    bool same = (int)total == b->S;
    for (int i = 0; same && i < b->n_scen; ++i) same = b->first[i + 1] - b->first[i] == counts[i];
    int rc;
    if (!same && (rc = set_entries(b, counts))) return rc;
    for (int i = 0; i < b->n_scen; ++i) {
        if (b->hyeto[i]) cudaFree(b->hyeto[i]);
        b->hyeto[i] = nullptr;
        BCK(b, cudaMalloc(&b->hyeto[i], sizeof(float) * std::max(1, n_blocks[i])));
        if (n_blocks[i] > 0)
            BCK(b, cudaMemcpy(b->hyeto[i], hyetographs[i], sizeof(float) * n_blocks[i], cudaMemcpyDefault));
    }
    std::vector<float> rm(b->S), sc(b->S);
    BCK(b, cudaMemcpy(rm.data(), rain_mult, sizeof(float) * b->S, cudaMemcpyDefault));
    BCK(b, cudaMemcpy(sc.data(), manning_scale, sizeof(float) * b->S, cudaMemcpyDefault));
    for (int e = 0; e < b->S; ++e) {
        const int i = b->scen_of[e];
        flood::ScenDesc& d = b->desc[e];
        d.hyeto = b->hyeto[i];
        d.nb = n_blocks[i];
        d.rain_mult = rm[e];
        d.scale = sc[e];
        d.t_end = t_end[i];
        for (int q = 0; q < 4; ++q) d.lc_n[q] = b->lc[i] ? b->lc_n0[i][q] : 0.0f;
        d.lc_drain = 0.0f;
        BCK(b, cudaMemsetAsync(b->state[e], 0, sizeof(float) * 6 * d.plane, s));
    }
    BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(flood::ScenDesc) * b->S,
                           cudaMemcpyHostToDevice, s));
    std::vector<MemberClock> ms((size_t)3 * b->S);
    for (auto& c : ms) { c.t = 0.0; c.steps = 0; c.hmax_bits = 0; c.cur = 0; }
    BCK(b, cudaMemcpyAsync(b->ms, ms.data(), sizeof(MemberClock) * 3 * b->S, cudaMemcpyHostToDevice, s));
    BCK(b, cudaMemsetAsync(b->rain_acc, 0, sizeof(double) * b->S, s));
    BCK(b, cudaMemsetAsync(b->vacc, 0, sizeof(double) * b->nslot * 2, s));
    BCK(b, cudaMemsetAsync(b->dacc, 0, sizeof(double) * std::max(b->nslot, 1), s));
    BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), s));
    BCK(b, cudaStreamSynchronize(s));
    b->k = 0;
    b->initialised = true;
    drop_graph(b);  // the launches depend on land cover being on
    return FLOOD_OK;
}

int flood_batch_init(flood_batch* b, const float* const* hyetographs, const int32_t* n_blocks,
                     const float* rain_mult, const float* manning_scale, const double* t_end,
                     void* stream)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    const std::vector<int32_t> ones(b->n_scen, 1);
    return flood_batch_init_members(b, hyetographs, n_blocks, ones.data(), rain_mult, manning_scale,
                                    t_end, stream);
}

int flood_batch_set_engine(flood_batch* b, int engine)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (engine < 0 || engine > 2) return bfail(b, FLOOD_ERR_ARG, "engine must be 0, 1 or 2");
    if (engine >= 1 && !b->d_maps) return bfail(b, FLOOD_ERR_STATE, "no tensor maps: direct loads only");
    if (engine == 2) {
        int dev = 0, coop = 0;
        BCK(b, cudaGetDevice(&dev));
        BCK(b, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (!coop) return bfail(b, FLOOD_ERR_STATE, "the device has no cooperative launch");
        if (!b->pbar) BCK(b, cudaMalloc(&b->pbar, sizeof(unsigned) * 4));
        if (!b->pact) BCK(b, cudaMalloc(&b->pact, sizeof(int) * 2));
        if (!b->pdone) BCK(b, cudaMalloc(&b->pdone, sizeof(int64_t)));
        if (!b->pdiag) BCK(b, cudaMalloc(&b->pdiag, sizeof(int) * 8));
    }
    BCK(b, cudaDeviceSynchronize());
    b->engine = engine;
    drop_graph(b);
    return FLOOD_OK;
}

int flood_batch_set_wait_budget(flood_batch* b, int64_t cycles)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    b->wait_budget = cycles < 0 ? -1 : (long long)cycles;
    return FLOOD_OK;
}

int flood_batch_set_launch(flood_batch* b, int rows_per_strip, int warps_per_cta)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (rows_per_strip < 1 || rows_per_strip > 4096 || (warps_per_cta != 4 && warps_per_cta != 8))
        return bfail(b, FLOOD_ERR_ARG, "rows_per_strip in [1, 4096], warps_per_cta 4 or 8");
    BCK(b, cudaDeviceSynchronize());
    // fold the volume slots of each scenario before the table changes
    std::vector<double> per((size_t)b->S * 2, 0.0), dper(b->S, 0.0);
    if (b->vacc && b->nslot) {
        std::vector<double> v((size_t)b->nslot * 2), dv(b->nslot);
        BCK(b, cudaMemcpy(v.data(), b->vacc, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
        BCK(b, cudaMemcpy(dv.data(), b->dacc, sizeof(double) * dv.size(), cudaMemcpyDeviceToHost));
        for (const auto& t : b->tasks) {
            per[(size_t)t.scen * 2] += v[(size_t)t.slot * 2];
            per[(size_t)t.scen * 2 + 1] += v[(size_t)t.slot * 2 + 1];
            dper[t.scen] += dv[t.slot];
        }
    }
    b->rows_per_strip = rows_per_strip;
    b->warps_per_cta = warps_per_cta;
    int rc = build_tasks(b);
    if (rc) return rc;
    return put_entry_sums(b, per, dper);
}

int flood_batch_step(flood_batch* b, double t_stop, void* stream)
{
    const flood::TraceRange range("flood_batch_step");
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (!b->initialised) return bfail(b, FLOOD_ERR_STATE, "flood_batch_init has not been called");
    if (!(t_stop >= 0.0)) return bfail(b, FLOOD_ERR_ARG, "t_stop must be >= 0");
    cudaStream_t s = S_(stream);
    int rc = b->engine == 2 ? FLOOD_OK : ensure_graph(b);
    if (rc) return rc;
    BCK(b, cudaMemcpyAsync(b->t_stop, &t_stop, sizeof(double), cudaMemcpyHostToDevice, s));
    std::vector<MemberClock> c;
    double last = -1.0;
    for (int rounds = 0;; ++rounds) {
        if ((rc = read_batch_clocks(b, c, s))) return rc;
        int64_t need = 0;
        double tmin = 1e300;
        for (int i = 0; i < b->S; ++i) {
            const double te = std::min(t_stop, b->desc[i].t_end);
            if (c[i].t >= te) continue;
            tmin = std::min(tmin, c[i].t);
            double dt;
            if (b->p.dt_fixed > 0) {
                dt = b->p.dt_fixed;
            } else {
                float hf;
                std::memcpy(&hf, &c[i].hmax_bits, sizeof(hf));
                const double hm = std::max((double)hf, b->p.h_floor);
                dt = std::min(b->p.alpha * b->p.dx / std::sqrt(b->p.g * hm), b->p.dt_cap);
            }
            const double rb = b->p.rain_block;
            const int64_t edges = (int64_t)std::floor(te / rb) - (int64_t)std::floor(c[i].t / rb) + 1;
            need = std::max(need, (int64_t)std::ceil((te - c[i].t) / dt) + edges);
        }
        if (need == 0) break;
        if (rounds > 0 && !(tmin > last))
            return bfail(b, FLOOD_ERR_STATE, "scenarios stopped advancing toward t_stop");
        if (need > (int64_t)1 << 26) return bfail(b, FLOOD_ERR_STATE, "too many steps to t_stop");
        last = tmin;
        if (b->engine == 2) {  // one persistent launch runs every scenario to the stop
            flood::PersistArgs q{};
            q.a = batch_args(b, 0);
            q.ms = b->ms;
            q.S = b->S;
            q.max_steps = (int)std::min<int64_t>(2 * need + 64, INT32_MAX / 2);
            q.k0 = b->k;
            q.bar = b->pbar;
            q.task_next = b->pbar + 2;
            q.any_active = b->pact;
            q.steps_done = b->pdone;
            q.budget = b->wait_budget < 0 ? flood::kTmaWaitBudgetDefault : b->wait_budget;
            q.diag = b->pdiag;
            BCK(b, cudaMemsetAsync(b->pdiag, 0, sizeof(int) * 8, s));
            BCK(b, cudaMemsetAsync(b->pbar, 0, sizeof(unsigned) * 4, s));
            BCK(b, cudaMemsetAsync(b->pact, 0, sizeof(int) * 2, s));
            BCK(b, flood::launch_batch_persistent(q, s));
            int64_t done = 0;
            BCK(b, cudaMemcpyAsync(&done, b->pdone, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            BCK(b, cudaStreamSynchronize(s));
            b->k += done;
            b->launches += 1;
            int dg[8];
            BCK(b, cudaMemcpy(dg, b->pdiag, sizeof(dg), cudaMemcpyDeviceToHost));
            if (dg[0])
                return bfail(b, FLOOD_ERR_TIMEOUT,
                             std::string(dg[0] == 1 ? "grid barrier" : "staged-row wait") +
                                 " gave up at step " + std::to_string(dg[1]) + " in CTA " +
                                 std::to_string(dg[2]) + " of " + std::to_string(dg[5]) + " (" +
                                 std::to_string(dg[3]) + ", " + std::to_string(dg[4]) + ")");
            continue;
        }
        const int64_t reps = (need + kGraphSteps - 1) / kGraphSteps;
        for (int64_t r = 0; r < reps; ++r) BCK(b, cudaGraphLaunch(b->graph, s));
        b->k += reps * kGraphSteps;
        b->launches += reps * kGraphSteps * 2;
    }
    return FLOOD_OK;
}

int flood_batch_get_member_state(flood_batch* b, int scen, int member, float* h, float* qx,
                                 float* qy, void* stream)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (scen < 0 || scen >= b->n_scen) return bfail(b, FLOOD_ERR_ARG, "scenario out of range");
    if (member < 0 || member >= b->first[scen + 1] - b->first[scen])
        return bfail(b, FLOOD_ERR_ARG, "member out of range");
    const int i = b->first[scen] + member;
    cudaStream_t s = S_(stream);
    MemberClock c;
    BCK(b, cudaMemcpyAsync(&c, b->ms + (b->k % 3) * b->S + i, sizeof(c), cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    const flood::ScenDesc& d = b->desc[i];
    const float* base = d.state + (size_t)c.cur * 3 * d.plane;
    float* outs[3] = {h, qx, qy};
    for (int k = 0; k < 3; ++k)
        if (outs[k])
            BCK(b, cudaMemcpy2DAsync(outs[k], sizeof(float) * d.nx, base + k * d.plane,
                                     sizeof(float) * d.ld, sizeof(float) * d.nx, d.ny,
                                     cudaMemcpyDefault, s));
    BCK(b, cudaStreamSynchronize(s));
    return FLOOD_OK;
}

int flood_batch_get_state(flood_batch* b, int i, float* h, float* qx, float* qy, void* stream)
{
    return flood_batch_get_member_state(b, i, 0, h, qx, qy, stream);
}

int flood_batch_members(flood_batch* b, double* t, int64_t* steps, double* storage, double* rain,
                        double* outflow, double* clamp)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    BCK(b, cudaDeviceSynchronize());
    std::vector<MemberClock> c(b->S);
    BCK(b, cudaMemcpy(c.data(), b->ms + (b->k % 3) * b->S, sizeof(MemberClock) * b->S,
                      cudaMemcpyDeviceToHost));
    for (int i = 0; i < b->S; ++i) {
        if (t) t[i] = c[i].t;
        if (steps) steps[i] = c[i].steps;
    }
    if (rain) BCK(b, cudaMemcpy(rain, b->rain_acc, sizeof(double) * b->S, cudaMemcpyDeviceToHost));
    if (outflow || clamp) {
        std::vector<double> v((size_t)b->nslot * 2);
        BCK(b, cudaMemcpy(v.data(), b->vacc, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
        std::vector<double> o(b->S, 0.0), cl(b->S, 0.0);
        for (const auto& tk : b->tasks) {
            o[tk.scen] += v[(size_t)tk.slot * 2];
            cl[tk.scen] += v[(size_t)tk.slot * 2 + 1];
        }
        for (int i = 0; i < b->S; ++i) {
            if (outflow) outflow[i] = o[i];
            if (clamp) clamp[i] = cl[i];
        }
    }
    if (storage) {
        for (int i = 0; i < b->S; ++i) {
            const flood::ScenDesc& d = b->desc[i];
            if (flood::launch_storage(d.state, b->ms + (b->k % 3) * b->S + i, 1, d.ny, d.nx, d.ld,
                                      d.plane, b->p.dx * b->p.dx, b->part, b->part_cap,
                                      b->storage + i, 0))
                return bfail(b, FLOOD_ERR_STATE, "storage partial buffer too small");
        }
        BCK(b, cudaGetLastError());
        BCK(b, cudaMemcpy(storage, b->storage, sizeof(double) * b->S, cudaMemcpyDeviceToHost));
    }
    return FLOOD_OK;
}

int64_t flood_batch_launch_count(const flood_batch* b) { return b ? b->launches : 0; }

int flood_batch_autotune(flood_batch* b, double trial_s, int* best_rows, int* best_warps,
                         int* best_engine, double* best_ms, void* stream)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (!b->initialised) return bfail(b, FLOOD_ERR_STATE, "flood_batch_init has not been called");
    if (!(trial_s > 0.0)) return bfail(b, FLOOD_ERR_ARG, "trial_s must be > 0");
    cudaStream_t s = S_(stream);
    const int S = b->S;
    BCK(b, cudaStreamSynchronize(s));
    // the batch as it is: clocks (all three slots), each scenario's current
    // state, rain and per-scenario volume sums
    std::vector<MemberClock> ms0((size_t)3 * S);
    BCK(b, cudaMemcpy(ms0.data(), b->ms, sizeof(MemberClock) * ms0.size(), cudaMemcpyDeviceToHost));
    const MemberClock* c0 = ms0.data() + (b->k % 3) * S;
    std::vector<double> rain0(S), per((size_t)S * 2, 0.0), dper(S, 0.0), v((size_t)b->nslot * 2),
        dv(std::max(b->nslot, 1));
    BCK(b, cudaMemcpy(rain0.data(), b->rain_acc, sizeof(double) * S, cudaMemcpyDeviceToHost));
    BCK(b, cudaMemcpy(v.data(), b->vacc, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
    BCK(b, cudaMemcpy(dv.data(), b->dacc, sizeof(double) * dv.size(), cudaMemcpyDeviceToHost));
    for (const auto& t : b->tasks) {
        per[(size_t)t.scen * 2] += v[(size_t)t.slot * 2];
        per[(size_t)t.scen * 2 + 1] += v[(size_t)t.slot * 2 + 1];
        dper[t.scen] += dv[t.slot];
    }
    size_t total = 0;
    for (int i = 0; i < S; ++i) total += 3 * b->desc[i].plane;
    float* snap = nullptr;
    BCK(b, cudaMalloc(&snap, sizeof(float) * total));
    auto copy_states = [&](bool save) -> cudaError_t {
        size_t off = 0;
        for (int i = 0; i < S; ++i) {
            const size_t n = 3 * b->desc[i].plane;
            float* cur = b->state[i] + (size_t)c0[i].cur * n;
            cudaError_t e = cudaMemcpyAsync(save ? snap + off : cur, save ? cur : snap + off,
                                            sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            off += n;
        }
        return cudaSuccess;
    };
    const int64_t k0 = b->k;
    // put the batch back as it was, in the current task layout
    auto restore = [&]() -> int {
        BCK(b, copy_states(false));
        BCK(b, cudaMemcpyAsync(b->ms, ms0.data(), sizeof(MemberClock) * ms0.size(),
                               cudaMemcpyHostToDevice, s));
        BCK(b, cudaMemcpyAsync(b->rain_acc, rain0.data(), sizeof(double) * S, cudaMemcpyHostToDevice, s));
        BCK(b, cudaStreamSynchronize(s));
        const int rc_sums = put_entry_sums(b, per, dper);
        if (rc_sums) return rc_sums;
        BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), s));
        BCK(b, cudaStreamSynchronize(s));
        b->k = k0;
        return FLOOD_OK;
    };
    int rc = FLOOD_OK;
    {
        const cudaError_t e = copy_states(true);
        if (e != cudaSuccess) {
            cudaFree(snap);
            return bfail(b, FLOOD_ERR_CUDA, std::string("snapshot: ") + cudaGetErrorString(e));
        }
    }
    double t_from = 0.0;
    for (int i = 0; i < S; ++i) t_from = std::max(t_from, std::min(c0[i].t, b->desc[i].t_end));
    const double t_trial = t_from + trial_s;
    struct Cand { int rows, warps, engine; };
    std::vector<Cand> cands;
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    for (int r : {16, 32, 64}) {
        if (b->d_maps) {
            cands.push_back({r, 4, 1});
            cands.push_back({r, 8, 1});
            if (coop) cands.push_back({r, 4, 2});
        } else {
            cands.push_back({r, 4, 0});
            cands.push_back({r, 8, 0});
        }
    }
    const int rows0 = b->rows_per_strip, warps0 = b->warps_per_cta, eng0 = b->engine;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    Cand bc{rows0, warps0, eng0};
    for (const Cand& cd : cands) {
        if ((rc = flood_batch_set_launch(b, cd.rows, cd.warps))) break;
        if ((rc = flood_batch_set_engine(b, cd.engine))) break;
        if ((rc = restore())) break;
        if ((rc = flood_batch_step(b, t_trial, stream))) break;  // warm-up: graph capture, caches
        if ((rc = restore())) break;
        cudaEventRecord(e0, s);
        if ((rc = flood_batch_step(b, t_trial, stream))) break;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) {
            best = t;
            bc = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc2 = flood_batch_set_launch(b, rc ? rows0 : bc.rows, rc ? warps0 : bc.warps);
    if (!rc2) rc2 = flood_batch_set_engine(b, rc ? eng0 : bc.engine);
    if (!rc2) rc2 = restore();
    cudaFree(snap);
    if (rc) return rc;
    if (rc2) return rc2;
    if (best_rows) *best_rows = bc.rows;
    if (best_warps) *best_warps = bc.warps;
    if (best_engine) *best_engine = bc.engine;
    if (best_ms) *best_ms = best;
    return FLOOD_OK;
}

// ---- land cover (Section 4.1) --------------------------------------------

int flood_batch_set_land_cover(flood_batch* b, int scen, const uint8_t* cls, int n_classes,
                               const flood_land_class* classes)
{
    constexpr float kWallZ = 1.0e6f;  // m: the bed of cells outside the domain
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (scen < 0 || scen >= b->n_scen) return bfail(b, FLOOD_ERR_ARG, "scenario out of range");
    if (b->initialised) return bfail(b, FLOOD_ERR_STATE, "land cover is set before flood_batch_init");
    if (b->lc[scen]) return bfail(b, FLOOD_ERR_STATE, "land cover is already set for the scenario");
    if (!cls || !classes || n_classes < 1 || n_classes > 4)
        return bfail(b, FLOOD_ERR_ARG, "need cls, 1..4 classes and their table");
    for (int q = 0; q < n_classes; ++q) {
        const flood_land_class& k = classes[q];
        if (!(k.n > 0.0f) || !(k.runoff >= 0.0f && k.runoff <= 1.0f) ||
            (k.drains != 0 && k.drains != 1) || (k.outside != 0 && k.outside != 1))
            return bfail(b, FLOOD_ERR_ARG, "class needs n > 0, runoff in [0, 1], flags 0/1");
    }
    const int ny = b->sny[scen], nx = b->snx[scen], ld = b->sld[scen];
    const size_t plane = (size_t)ny * ld;
    std::vector<uint8_t> hc((size_t)ny * nx);
    BCK(b, cudaMemcpy(hc.data(), cls, hc.size(), cudaMemcpyDefault));
    std::array<float, 4> runoff{1.0f, 1.0f, 1.0f, 1.0f}, drains{0.0f, 0.0f, 0.0f, 0.0f},
        n0{0.05f, 0.05f, 0.05f, 0.05f};
    for (int q = 0; q < n_classes; ++q) {
        runoff[q] = classes[q].outside ? 0.0f : classes[q].runoff;
        drains[q] = classes[q].outside ? 0.0f : (float)classes[q].drains;
        n0[q] = classes[q].n;
    }
    const int spans = (nx + kSpan - 1) / kSpan;
    std::vector<uint8_t> pad(plane, 0), span_out((size_t)ny * spans, 1);
    std::vector<float> z(plane);
    BCK(b, cudaMemcpy(z.data(), b->zn[scen], sizeof(float) * plane, cudaMemcpyDeviceToHost));
    double rain_cells = 0.0;
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < nx; ++c) {
            const uint8_t k = hc[(size_t)r * nx + c];
            if (k >= n_classes) return bfail(b, FLOOD_ERR_ARG, "class index out of range");
            pad[(size_t)r * ld + c] = k;
            rain_cells += runoff[k];
            if (classes[k].outside)
                z[(size_t)r * ld + c] = kWallZ;  // no link into the cell carries flow (Eq. 3)
            else
                span_out[(size_t)r * spans + c / kSpan] = 0;
        }
    uint8_t* d_cls = nullptr;
    float* d_zc = nullptr;
    BCK(b, cudaMalloc(&d_cls, plane));
    cudaError_t e = cudaMalloc(&d_zc, sizeof(float) * 2 * plane);
    if (e != cudaSuccess) {
        cudaFree(d_cls);
        BCK(b, e);
    }
    b->cls8[scen] = d_cls;
    b->zc[scen] = d_zc;
    BCK(b, cudaMemcpy(d_cls, pad.data(), plane, cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(b->zn[scen], z.data(), sizeof(float) * plane, cudaMemcpyHostToDevice));
    // the TMA engines' static planes: the bed and each cell's class code
    // where the roughness plane would be
    std::vector<uint32_t> codes(plane);
    for (size_t i = 0; i < plane; ++i) codes[i] = pad[i];
    BCK(b, cudaMemcpy(d_zc, z.data(), sizeof(float) * plane, cudaMemcpyHostToDevice));
    BCK(b, cudaMemcpy(d_zc + plane, codes.data(), sizeof(uint32_t) * plane, cudaMemcpyHostToDevice));
    b->lc_K[scen] = n_classes;
    b->lc_runoff[scen] = runoff;
    b->lc_drains[scen] = drains;
    b->lc_n0[scen] = n0;
    b->lc_rain_cells[scen] = rain_cells;
    b->span_out[scen] = std::move(span_out);
    b->lc[scen] = 1;
    std::vector<int> counts(b->n_scen);
    for (int i = 0; i < b->n_scen; ++i) counts[i] = b->first[i + 1] - b->first[i];
    return set_entries(b, counts);
}

int flood_batch_set_land_params(flood_batch* b, int scen, const float* n_class,
                                const float* drain_rate)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (scen < 0 || scen >= b->n_scen) return bfail(b, FLOOD_ERR_ARG, "scenario out of range");
    if (!b->initialised || !b->lc[scen])
        return bfail(b, FLOOD_ERR_STATE, "needs land cover and flood_batch_init");
    const int e0 = b->first[scen], N = b->first[scen + 1] - e0, K = b->lc_K[scen];
    BCK(b, cudaDeviceSynchronize());
    if (n_class) {
        std::vector<float> in((size_t)N * K);
        BCK(b, cudaMemcpy(in.data(), n_class, sizeof(float) * in.size(), cudaMemcpyDefault));
        for (float v : in)
            if (!(v > 0.0f) || !std::isfinite(v))
                return bfail(b, FLOOD_ERR_ARG, "class roughness must be positive");
        for (int m = 0; m < N; ++m)
            for (int q = 0; q < K; ++q) b->desc[e0 + m].lc_n[q] = in[(size_t)m * K + q];
    }
    if (drain_rate) {
        std::vector<float> d(N);
        BCK(b, cudaMemcpy(d.data(), drain_rate, sizeof(float) * N, cudaMemcpyDefault));
        for (float v : d)
            if (!(v >= 0.0f) || !std::isfinite(v))
                return bfail(b, FLOOD_ERR_ARG, "drainage rates must be >= 0");
        for (int m = 0; m < N; ++m) b->desc[e0 + m].lc_drain = d[m];
    }
    BCK(b, cudaMemcpy(b->d_desc + e0, b->desc.data() + e0, sizeof(flood::ScenDesc) * N,
                      cudaMemcpyHostToDevice));
    return FLOOD_OK;
}

int flood_batch_drained_volume(flood_batch* b, double* drained)
{
    if (!b) return bfail(nullptr, FLOOD_ERR_ARG, "batch is NULL");
    if (!drained) return bfail(b, FLOOD_ERR_ARG, "drained is NULL");
    BCK(b, cudaDeviceSynchronize());
    std::vector<double> dv(std::max(b->nslot, 1)), out(b->S, 0.0);
    BCK(b, cudaMemcpy(dv.data(), b->dacc, sizeof(double) * dv.size(), cudaMemcpyDeviceToHost));
    for (const auto& t : b->tasks) out[t.scen] += dv[t.slot];
    std::copy(out.begin(), out.end(), drained);
    return FLOOD_OK;
}

}  // extern "C"
