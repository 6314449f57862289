// flood_adjoint: gradients of a gauge-misfit loss by reverse mode with
// checkpointing (extension beyond the paper).  Forward: the ensemble advances
// through the observation times exactly as flood_step would, logging each
// member's step lengths and storing its state every ckpt_every steps.
// Reverse: segment by segment from the last, the segment's states are
// recomputed bit for bit from its checkpoint (replay kernel), then the
// adjoint kernel runs backwards through them, seeded with the loss
// sensitivities at the observation times.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "adjoint.cuh"
#include "tma.cuh"
#include "grid.cuh"
#include "pf_kernels.cuh"

using flood::MemberClock;
#define CK FLOOD_CK

namespace {

cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <class T>
int grow(flood_grid* g, T** p, size_t& have, size_t count)
{
    if (*p && have >= count) return FLOOD_OK;
    have = count;
    return flood::dalloc(g, p, count);
}

// Put the state saved in ckpt slot 0 back into each member's current buffer
// and restore the saved clocks and volume counters (a forward that overflowed
// the step log is redone).
int restore_start(flood_grid* g, const std::vector<MemberClock>& c0, const std::vector<double>& rain0,
                  const std::vector<double>& vacc0, cudaStream_t s)
{
    const int M = g->M;
    const size_t ms = 3 * g->plane;
    std::vector<MemberClock> now;
    int rc = flood::read_clocks(g, now, s);
    if (rc) return rc;
    std::vector<MemberClock> back = c0;
    for (int m = 0; m < M; ++m) {
        back[m].cur = now[m].cur;
        back[m].steps = 0;
        CK(g, cudaMemcpyAsync(g->state + (size_t)(now[m].cur * M + m) * ms, g->ckpt + (size_t)m * ms,
                              sizeof(float) * ms, cudaMemcpyDeviceToDevice, s));
    }
    CK(g, cudaMemcpyAsync(g->ms + (g->k % 3) * M, back.data(), sizeof(MemberClock) * M,
                          cudaMemcpyHostToDevice, s));
    CK(g, cudaMemcpyAsync(g->rain_acc, rain0.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
    CK(g, cudaMemcpyAsync(g->vacc, vacc0.data(), sizeof(double) * vacc0.size(), cudaMemcpyHostToDevice, s));
    CK(g, cudaStreamSynchronize(s));
    return FLOOD_OK;
}

}  // namespace

extern "C" int flood_adjoint(flood_grid* g, const flood_loss_spec* L, int ckpt_every, float* grad_n,
                             double* grad_rain, double* grad_scale, float* grad_h0, double* loss_out,
                             void* stream)
{
    const flood::TraceRange range("flood_adjoint");
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (g->M == 0) return flood::fail(g, FLOOD_ERR_STATE, "flood_ensemble_init has not been called");
    if (!L || L->n_samples < 1 || !(L->sample_dt > 0) || L->n_gauges < 1 || !L->cells || !L->d)
        return flood::fail(g, FLOOD_ERR_ARG, "invalid flood_loss_spec");
    if (ckpt_every < 0) return flood::fail(g, FLOOD_ERR_ARG, "ckpt_every must be >= 0");
    cudaStream_t s = S(stream);
    const int M = g->M, ns = L->n_samples, G = L->n_gauges;
    const size_t ms = 3 * g->plane;

    std::vector<MemberClock> c0;
    int rc = flood::read_clocks(g, c0, s);
    if (rc) return rc;
    const double t0 = c0[0].t;
    for (int m = 1; m < M; ++m)
        if (c0[m].t != t0) return flood::fail(g, FLOOD_ERR_STATE, "members are not at the same time");
    std::vector<int32_t> cells(G);
    std::vector<double> d((size_t)ns * G);
    CK(g, cudaMemcpy(cells.data(), L->cells, sizeof(int32_t) * G, cudaMemcpyDefault));
    CK(g, cudaMemcpy(d.data(), L->d, sizeof(double) * ns * G, cudaMemcpyDefault));
    for (int k = 0; k < G; ++k)
        if (cells[k] < 0 || (int64_t)cells[k] >= (int64_t)g->ny * g->nx)
            return flood::fail(g, FLOOD_ERR_ARG, "gauge cell index out of range");

    // saved start: clocks, volume counters (restored if the forward is redone)
    std::vector<double> rain0(M), vacc0((size_t)M * g->nslot * 2);
    CK(g, cudaMemcpy(rain0.data(), g->rain_acc, sizeof(double) * M, cudaMemcpyDeviceToHost));
    CK(g, cudaMemcpy(vacc0.data(), g->vacc, sizeof(double) * vacc0.size(), cudaMemcpyDeviceToHost));

    const double T = ns * L->sample_dt;
    const double dt_ref = g->p.dt_fixed > 0 ? g->p.dt_fixed : g->p.dt_cap;
    int cap = (int)std::ceil(T / dt_ref) + 2 * ns + 8;
    std::vector<int64_t> steps0(M);
    for (int m = 0; m < M; ++m) steps0[m] = c0[m].steps;
    std::vector<int> K_m(M);
    std::vector<int32_t> samp_step((size_t)ns * M);
    size_t have_ckpt = 0, have_log = 0, have_sy = 0;
    int K = 0;
    cudaEvent_t e0, e1, e2;
    CK(g, cudaEventCreate(&e0));
    CK(g, cudaEventCreate(&e1));
    CK(g, cudaEventCreate(&e2));
    for (int attempt = 0;; ++attempt) {
        K = ckpt_every > 0 ? ckpt_every : std::max(1, (int)std::lround(std::sqrt((double)cap)));
        const size_t n_ckpt = (size_t)cap / K + 1;
        have_log = 0;
        if ((rc = grow(g, &g->log, have_log, (size_t)M * cap))) return rc;
        if (n_ckpt * M * ms > g->ckpt_floats) {
            have_ckpt = 0;
            if ((rc = grow(g, &g->ckpt, have_ckpt, n_ckpt * M * ms))) return rc;
            g->ckpt_floats = n_ckpt * M * ms;
        }
        have_sy = 0;
        if ((rc = grow(g, &g->samp_y, have_sy, (size_t)ns * M * G))) return rc;
        g->log_cap = cap;
        g->ckpt_every = K;
        // checkpoint 0: the starting state; clocks count steps from 0
        std::vector<MemberClock> cz;
        if ((rc = flood::read_clocks(g, cz, s))) return rc;
        for (int m = 0; m < M; ++m) {
            CK(g, cudaMemcpyAsync(g->ckpt + (size_t)m * ms, g->state + (size_t)(cz[m].cur * M + m) * ms,
                                  sizeof(float) * ms, cudaMemcpyDeviceToDevice, s));
            cz[m].steps = 0;
        }
        CK(g, cudaMemcpyAsync(g->ms + (g->k % 3) * M, cz.data(), sizeof(MemberClock) * M,
                              cudaMemcpyHostToDevice, s));
        g->logging = true;
        CK(g, cudaEventRecord(e0, s));
        int64_t kmax = 0;
        for (int sidx = 1; sidx <= ns; ++sidx) {
            rc = flood_step(g, 0, t0 + sidx * L->sample_dt, stream);
            if (rc) {
                g->logging = false;
                return rc;
            }
            // the cells live in samp_cells (device) for both gauge sampling and seeding
            if (sidx == 1) {
                size_t hc = 0;
                if ((rc = grow(g, &g->samp_cells, hc, G))) return rc;
                CK(g, cudaMemcpyAsync(g->samp_cells, cells.data(), sizeof(int32_t) * G,
                                      cudaMemcpyHostToDevice, s));
            }
            flood::launch_gauge(g->state, g->ms + (g->k % 3) * M, g->samp_cells, G, M, g->ld, g->nx,
                                g->plane, g->samp_y + (size_t)(sidx - 1) * M * G, s);
            g->launches++;
            std::vector<MemberClock> cc;
            if ((rc = flood::read_clocks(g, cc, s))) {
                g->logging = false;
                return rc;
            }
            for (int m = 0; m < M; ++m) {
                samp_step[(size_t)(sidx - 1) * M + m] = (int32_t)cc[m].steps;
                K_m[m] = (int)std::min<int64_t>(cc[m].steps, INT32_MAX);
                kmax = std::max<int64_t>(kmax, cc[m].steps);
            }
        }
        CK(g, cudaEventRecord(e1, s));
        g->logging = false;
        if (kmax <= cap) break;
        if (attempt >= 4) return flood::fail(g, FLOOD_ERR_STATE, "step log could not hold the window");
        if ((rc = restore_start(g, c0, rain0, vacc0, s))) return rc;
        cap = (int)std::min<int64_t>((int64_t)kmax * 2 + 8, INT32_MAX / 2);
    }

    // loss per member from the recorded gauge outputs
    std::vector<float> yh((size_t)ns * M * G);
    CK(g, cudaMemcpy(yh.data(), g->samp_y, sizeof(float) * yh.size(), cudaMemcpyDeviceToHost));
    if (loss_out)
        for (int m = 0; m < M; ++m) {
            double acc = 0.0;
            for (int si = 0; si < ns; ++si)
                for (int k = 0; k < G; ++k) {
                    const double e = (double)yh[((size_t)si * M + m) * G + k] - d[(size_t)si * G + k];
                    acc += e * e;
                }
            loss_out[m] = acc;
        }

    // reverse sweep buffers
    size_t have = 0;
    if ((size_t)(K + 1) * M * ms > g->seg_floats) {
        if ((rc = grow(g, &g->seg, have, (size_t)(K + 1) * M * ms))) return rc;
        g->seg_floats = (size_t)(K + 1) * M * ms;
    }
    have = 0;
    if ((rc = grow(g, &g->lam, have, 2 * (size_t)M * ms))) return rc;
    have = 0;
    if ((rc = grow(g, &g->gpart, have, (size_t)M * g->nslot * 2))) return rc;
    have = 0;
    if ((rc = grow(g, &g->seg_end, have, M))) return rc;
    have = 0;
    if ((rc = grow(g, &g->samp_step, have, (size_t)ns * M))) return rc;
    have = 0;
    if ((rc = grow(g, &g->samp_d, have, (size_t)ns * G))) return rc;
    if (grad_n) {
        have = 0;
        if ((rc = grow(g, &g->gnm, have, (size_t)M * g->plane))) return rc;
        have = 0;
        if ((rc = grow(g, &g->gn_out, have, (size_t)g->ny * g->nx))) return rc;
        CK(g, cudaMemsetAsync(g->gnm, 0, sizeof(float) * M * g->plane, s));
    }
    CK(g, cudaMemsetAsync(g->lam, 0, sizeof(float) * 2 * M * ms, s));
    CK(g, cudaMemsetAsync(g->gpart, 0, sizeof(double) * M * g->nslot * 2, s));
    if (g->lc_on) {
        have = 0;
        if ((rc = grow(g, &g->gdpart, have, (size_t)M * g->nslot))) return rc;
        CK(g, cudaMemsetAsync(g->gdpart, 0, sizeof(double) * M * g->nslot, s));
    }
    CK(g, cudaMemcpyAsync(g->samp_step, samp_step.data(), sizeof(int32_t) * ns * M,
                          cudaMemcpyHostToDevice, s));
    CK(g, cudaMemcpyAsync(g->samp_d, d.data(), sizeof(double) * ns * G, cudaMemcpyHostToDevice, s));

    // land cover: each member's Manning n field and the share of the rain
    // that stays, from the classes (the step looks them up per cell)
    const size_t plane = g->plane;
    if (g->lc_on && (rc = flood::land_adjoint_fields(g, s))) return rc;

    // tensor maps of the TMA-staged replay and reverse stencil (direct loads
    // otherwise); short strips never fill the reverse stencil's copy
    // pipeline, so those keep its direct-load form
    flood::AdjTmaArgs tma{};
    bool use_tma = g->engine == 1 && g->maps_ok;
    if (use_tma) {
        const int bc = flood::adjoint_tma_box_cols();
        const uint64_t s1 = sizeof(float) * g->ld, s2 = sizeof(float) * g->plane;
        use_tma =
            flood::encode_map_3d(&tma.seg_map, g->seg, g->ld, g->ny, (uint64_t)(K + 1) * M * 3, s1,
                                 s2, bc, 1, 3) == 0 &&
            flood::encode_map_3d(&tma.seg1_map, g->seg, g->ld, g->ny, (uint64_t)(K + 1) * M * 3, s1,
                                 s2, bc, 1, 1) == 0 &&
            flood::encode_map_3d(&tma.lam_map, g->lam, g->ld, g->ny, (uint64_t)2 * M * 3, s1, s2, bc,
                                 1, 3) == 0 &&
            (!grad_n || flood::encode_map_3d(&tma.gn_map, g->gnm, g->ld, g->ny, (uint64_t)M, s1, s2,
                                             bc, 1, 1) == 0);
        // with land cover the bed and the class codes, as the forward stages them
        tma.static_map = g->lc_on ? g->static_map_lc : g->static_map;
    }
    const bool tma_replay = use_tma;
    const bool tma_reverse = use_tma && g->rows_per_strip >= 16;

    const int kmax = *std::max_element(K_m.begin(), K_m.end());
    const int n_seg = (kmax + K - 1) / K;
    int lam_in = 0;
    std::vector<int> seg_end(M);
    for (int cs = n_seg - 1; cs >= 0; --cs) {
        const int first = cs * K;
        int len = 0;
        for (int m = 0; m < M; ++m) {
            seg_end[m] = std::min(first + K, K_m[m]);
            len = std::max(len, seg_end[m] - first);
        }
        if (len <= 0) continue;
        CK(g, cudaMemcpyAsync(g->seg_end, seg_end.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s));
        CK(g, cudaMemcpyAsync(g->seg, g->ckpt + (size_t)cs * M * ms, sizeof(float) * M * ms,
                              cudaMemcpyDeviceToDevice, s));
        flood::StepArgs a = flood::step_args(g, -1.0);
        a.log = g->log;
        a.dt_log_cap = g->log_cap;
        a.ckpt = nullptr;
        a.seg = g->seg;
        a.seg_end = g->seg_end;
        a.seg_first = first;
        flood::TmaArgs rt;
        if (tma_replay) {
            rt.state_map = tma.seg_map;
            rt.static_map = g->lc_on ? g->static_map_lc : g->static_map;
        }
        for (int i = 0; i < len; ++i) {
            a.replay_i = i;
            if (tma_replay) {
                rt.a = a;
                flood::launch_replay_tma(rt, g->members_per_cta, s);
            } else {
                flood::launch_replay(a, g->members_per_cta, s);
            }
            g->launches++;
        }
        flood::AdjArgs b{};
        b.seg = g->seg;
        b.lam = g->lam;
        b.gn = grad_n ? g->gnm : nullptr;
        b.gpart = g->gpart;
        b.z = g->z;
        b.n = g->lc_on ? g->lc_adj + plane : g->n;
        b.n_mstride = g->lc_on ? plane : 0;
        b.rw = g->lc_on ? g->lc_adj + (size_t)(M + 1) * plane : nullptr;
        b.dflag = g->lc_on ? g->lc_adj + (size_t)(M + 2) * plane : nullptr;
        b.gdpart = g->lc_on ? g->gdpart : nullptr;
        if (g->lc_on) {
            b.lc_n = g->lc_n;
            for (int q = 0; q < 4; ++q) {
                b.lc_runoff[q] = g->lc_runoff[q];
                b.lc_drains[q] = g->lc_drains[q];
            }
        }
        b.scale = g->scale;
        b.log = g->log;
        b.seg_end = g->seg_end;
        b.dt_log_cap = g->log_cap;
        b.seg_first = first;
        b.plane = g->plane;
        b.ny = g->ny; b.nx = g->nx; b.ld = g->ld; b.M = M;
        b.rows_per_strip = g->rows_per_strip;
        b.nslot = g->nslot;
        b.g = g->p.g;
        b.dxd = g->p.dx;
        b.h_eps = (float)g->p.h_eps;
        b.edge_drop = (float)(g->p.edge_slope * g->p.dx);
        b.limiter = g->p.limiter;
        b.east_out = g->p.east_outflow;
        b.south_out = g->p.south_outflow;
        b.err = g->err;
        for (int i = 0; i < len; ++i) {
            b.rev_i = i;
            b.lam_in = lam_in;
            flood::launch_seed(b, g->samp_step, g->samp_y, g->samp_d, g->samp_cells, ns, G, s);
            if (tma_reverse) {
                tma.a = b;
                flood::launch_adjoint_tma(tma, g->members_per_cta, s);
            } else {
                flood::launch_adjoint(b, g->members_per_cta, s);
            }
            g->launches += 2;
            lam_in = 1 - lam_in;
        }
        CK(g, cudaGetLastError());
    }
    CK(g, cudaEventRecord(e2, s));
    CK(g, cudaStreamSynchronize(s));
    if ((rc = flood::check_err(g))) return rc;
    float fms = 0.0f, rms = 0.0f;
    cudaEventElapsedTime(&fms, e0, e1);
    cudaEventElapsedTime(&rms, e1, e2);
    g->adj_fwd_ms = fms;
    g->adj_rev_ms = rms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);

    if (grad_h0)
        for (int m = 0; m < M; ++m)
            CK(g, cudaMemcpy2DAsync(grad_h0 + (size_t)m * g->ny * g->nx, sizeof(float) * g->nx,
                                    g->lam + ((size_t)lam_in * M + m) * ms, sizeof(float) * g->ld,
                                    sizeof(float) * g->nx, g->ny, cudaMemcpyDefault, s));
    if (grad_n) {
        flood::launch_reduce_members(g->gnm, M, g->ny, g->nx, g->ld, g->plane, g->gn_out, s);
        g->launches++;
        CK(g, cudaMemcpyAsync(grad_n, g->gn_out, sizeof(float) * g->ny * g->nx, cudaMemcpyDefault, s));
    }
    if (grad_rain || grad_scale) {
        std::vector<double> gp((size_t)M * g->nslot * 2);
        CK(g, cudaMemcpyAsync(gp.data(), g->gpart, sizeof(double) * gp.size(), cudaMemcpyDeviceToHost, s));
        CK(g, cudaStreamSynchronize(s));
        for (int m = 0; m < M; ++m) {
            double gr = 0.0, gs = 0.0;
            for (int k = 0; k < g->nslot; ++k) {
                gr += gp[((size_t)m * g->nslot + k) * 2];
                gs += gp[((size_t)m * g->nslot + k) * 2 + 1];
            }
            if (grad_rain) grad_rain[m] = gr;
            if (grad_scale) grad_scale[m] = gs;
        }
    }
    g->adj_gdrain.assign(M, 0.0);
    if (g->lc_on) {
        std::vector<double> gp((size_t)M * g->nslot);
        CK(g, cudaMemcpyAsync(gp.data(), g->gdpart, sizeof(double) * gp.size(), cudaMemcpyDeviceToHost, s));
        CK(g, cudaStreamSynchronize(s));
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < g->nslot; ++k) g->adj_gdrain[m] += gp[(size_t)m * g->nslot + k];
    }
    // clocks keep counting from where they were
    std::vector<MemberClock> ce;
    if ((rc = flood::read_clocks(g, ce, s))) return rc;
    for (int m = 0; m < M; ++m) ce[m].steps += steps0[m];
    CK(g, cudaMemcpyAsync(g->ms + (g->k % 3) * M, ce.data(), sizeof(MemberClock) * M,
                          cudaMemcpyHostToDevice, s));
    CK(g, cudaStreamSynchronize(s));
    // what a calibration step may use: the gradients of this ensemble as it is now
    g->adj_epoch = g->epoch;
    g->adj_gn = grad_n != nullptr;
    g->adj_ns = ns;
    g->adj_G = G;
    g->adj_nslot = g->nslot;
    return FLOOD_OK;
}

extern "C" int flood_adjoint_timing(const flood_grid* g, double* forward_ms, double* reverse_ms)
{
    if (!g) return flood::fail(nullptr, FLOOD_ERR_ARG, "grid is NULL");
    if (forward_ms) *forward_ms = g->adj_fwd_ms;
    if (reverse_ms) *reverse_ms = g->adj_rev_ms;
    return FLOOD_OK;
}
