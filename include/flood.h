/*
 * flood.h -- C ABI of libflood.so, the GB300 (sm_103a) ensemble
 * local-inertial flood model with an on-device particle filter.
 *
 * Method: Wei et al., "Enable high-resolution, real-time ensemble simulation
 * and data assimilation of flood inundation using distributed GPU
 * parallelization" (arXiv 2302.08341).
 *
 * Conventions shared by every entry point
 *  - Return value: FLOOD_OK (0) or a negative FLOOD_ERR_* code.  After an
 *    error, flood_last_error(grid) returns a message (a static message for
 *    errors raised before a grid exists: flood_last_error(NULL)).
 *  - Grid: ny rows x nx columns of square cells of side dx.  Row-major
 *    arrays [ny][nx]; flat cell index = r * nx + c.  x runs along columns,
 *    y along rows.
 *  - Links (the paper's Lx / Ly, Section 3.1): qx[r][c] is the flow per unit
 *    width (m^2/s) on the link east of cell (r,c), positive toward +c;
 *    qy[r][c] is the link south of cell (r,c), positive toward +r.  The west
 *    and north edges are closed walls; qx[r][nx-1] / qy[ny-1][c] are the
 *    east / south edge links (zero unless that edge is a free outflow).
 *  - Pointers may be host or device memory (unified addressing decides);
 *    inputs are copied during the call, so the caller keeps ownership.
 *    Host outputs are complete when the call returns only for calls that
 *    are documented as synchronous; otherwise they are valid once `stream`
 *    has been synchronised.  Use page-locked host memory for overlap.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Work of one
 *    grid must be issued to one stream at a time.
 *  - Precision: state (h, qx, qy) and fields are FP32; time, time step,
 *    volume bookkeeping and particle weights are FP64.
 *  - The library owns every device buffer it allocates; flood_destroy frees
 *    them.
 */
#ifndef FLOOD_H
#define FLOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FLOOD_OK = 0,
    FLOOD_ERR_ARG = -1,      /* invalid argument (size, pointer, range)        */
    FLOOD_ERR_CUDA = -2,     /* a CUDA runtime call failed                     */
    FLOOD_ERR_OOM = -3,      /* device allocation failed                       */
    FLOOD_ERR_TIMEOUT = -4,  /* a bounded device wait (staged tiles) gave up    */
    FLOOD_ERR_NAN = -5,      /* a kernel produced a non-finite depth           */
    FLOOD_ERR_STATE = -6     /* call out of order (e.g. step before init)      */
};

typedef struct flood_grid flood_grid;

/* Scheme constants (Section 2.1, Section 4.1). */
typedef struct {
    double dx;          /* cell size, dx = dy (m); the paper's case uses 3 m         */
    double g;           /* gravitational acceleration, 9.81 m s^-2                   */
    double alpha;       /* Courant coefficient k of Eq. 4 (0.2..0.7; default 0.7)    */
    double dt_cap;      /* upper bound on the time step (s), default 1.0             */
    double dt_fixed;    /* > 0: fixed time step (the paper ran 0.25 s), else Eq. 4   */
    double h_eps;       /* links whose flow depth (Eq. 3) is <= h_eps carry no flow;
                           default 0: Eq. 2-3 as printed (no flow only at zero
                           flow depth).  A positive threshold makes FP32 and
                           FP64 runs part where depths cross it               */
    double h_floor;     /* floor on h_max inside Eq. 4 (m), default 1e-6             */
    double rain_block;  /* rain is piecewise constant over blocks of this length (s),
                           step (I) of Section 3.1: 300 s                          */
    double edge_slope;  /* bed slope continued past a free-outflow edge             */
    int32_t limiter;    /* 1: each link moves at most a quarter of the upstream
                           cell's volume per step (keeps depths non-negative)       */
    int32_t east_outflow;   /* 1: the east edge (c = nx-1) is a free outflow       */
    int32_t south_outflow;  /* 1: the south edge (r = ny-1) is a free outflow      */
    int32_t reserved;       /* must be 0                                           */
} flood_params;

/* Fill p with the defaults listed above (dx = 3, east free outflow). */
void flood_default_params(flood_params* p);

/* Message of the last error on grid g (or of the last error raised before a
 * grid existed, when g is NULL).  The string is owned by the library. */
const char* flood_last_error(const flood_grid* g);

/*
 * flood_create_grid -- the definitive (shared) data of the model: bed
 * elevation z and base Manning n, both [ny][nx] FP32 (Section 3.2: stored
 * once and shared by every member).  z should be referenced near 0 (its FP32
 * spacing bounds depth resolution).  Synchronous.
 * Errors: FLOOD_ERR_ARG for ny/nx < 1, NULL arrays, non-positive dx, g,
 * dt_cap or rain_block; FLOOD_ERR_OOM; FLOOD_ERR_CUDA.
 */
int flood_create_grid(flood_grid** out, int ny, int nx, const float* z, const float* n_base,
                      const flood_params* p);

/* Release every device buffer of g.  Safe on NULL.  Synchronous. */
int flood_destroy(flood_grid* g);

/*
 * flood_ensemble_init -- the initial ensemble (Eq. 6-7): N = n_members
 * particles with equal weights 1/N, each with its own state, rainfall
 * multiplier and Manning scale (the uncertain inputs, Section 4.1).
 *   h0            NULL (dry start), [ny][nx] shared by all members
 *                 (h0_per_member = 0) or [N][ny][nx] (h0_per_member = 1)
 *   rain_mult     [N] multiplier on the hyetograph
 *   manning_scale [N] multiplier on the base Manning field
 *   hyetograph    [n_blocks] rain rate (m/s) of each block of rain_block s
 *   t0            start time (s) of every member
 * Link fluxes start at zero.  (Re)allocates the ensemble buffers.
 * Synchronous.  Errors: FLOOD_ERR_ARG, FLOOD_ERR_OOM, FLOOD_ERR_CUDA.
 */
int flood_ensemble_init(flood_grid* g, int n_members, const float* h0, int h0_per_member,
                        const float* rain_mult, const float* manning_scale,
                        const float* hyetograph, int n_blocks, double t0, void* stream);

/*
 * flood_step -- evolve every member, x_{i,t+dt} = f(x_i, u_i, p_i) (Eq. 6),
 * with the local-inertial scheme of Section 2.1: link fluxes from Eq. 2-3,
 * then the continuity update of Eq. 5 and Eq. 1 with the block's rain, each
 * member with its own time step from Eq. 4 (CFL on the member's own maximum
 * depth), landing exactly on every rain-block edge and on t_end.
 *   t_end < 0   issue exactly n_steps steps (asynchronous).
 *   t_end >= 0  advance every member to t_end (members already there stay
 *               put).  n_steps <= 0: no limit on steps, > 0: at most n_steps
 *               steps.  Synchronises `stream` to follow the members' clocks.
 * Each step is a plan kernel then a step kernel on `stream`; with
 * flood_set_graphs, runs of 24 steps are replayed from a CUDA graph instead.
 * Errors: FLOOD_ERR_STATE before flood_ensemble_init, FLOOD_ERR_NAN if a
 * depth became non-finite (detected at the synchronisation points),
 * FLOOD_ERR_CUDA.
 */
int flood_step(flood_grid* g, int n_steps, double t_end, void* stream);

/*
 * flood_gauge_sample -- DA step (I) of Section 3.3: model output of every
 * member at the gauges, y[i][k] = depth of member i at flat cell
 * cell_idx[k].  y_out: [N][n_gauges] FP32 (host or device, may be NULL).
 * The sample is also kept on the device as the default input of
 * pf_assimilate.  Asynchronous.  Errors: FLOOD_ERR_ARG for a cell index out
 * of range or n_gauges < 1.
 */
int flood_gauge_sample(flood_grid* g, int n_gauges, const int32_t* cell_idx, float* y_out,
                       void* stream);

/*
 * pf_assimilate -- DA steps (II)-(V) of Section 3.3 on the device:
 *   weights   w_i+ proportional to p(d|x_i) w_i- (Eq. 9-11) with the diagonal
 *             Gaussian likelihood of Eq. 9 (sigma[k] absolute, or
 *             sigma_rel * d[k] when sigma_rel > 0 as in Section 4.4), formed
 *             in FP64 log-sum-exp;
 *   N_eff     = 1 / sum w_i^2 (Eq. 12);
 *   resample  if N_eff < n_thr_frac * N (Section 3.3 uses 0.8) or
 *             force_resample: systematic resampling (Arulampalam et al. 2002)
 *             with offsets (u + j)/N, u in [0,1) supplied by the caller;
 *             survivors keep their slot, the extra copies of each particle
 *             (in particle order) overwrite the dropped particles' slots (in
 *             slot order); every member's rain multiplier is then multiplied
 *             by beta[i] (Section 4.4: beta ~ N(1, 0.05^2), drawn by the
 *             caller) and the weights reset to 1/N.
 *   y            [N][n_gauges] FP32 model outputs or NULL = last gauge sample
 *   d, sigma     [n_gauges] FP64 observations and their standard deviations
 *   beta         [N] FP32 (only read when resampling)
 *   weights_out  [N] FP64 posterior weights before any reset (or NULL)
 *   idx_out      [N] int32 resampled particle indices, non-decreasing; the
 *                identity 0..N-1 when no resampling happened (or NULL)
 *   neff_out     N_eff, or 0 when every posterior weight underflowed to zero
 *                (the ensemble is then left unchanged) (or NULL)
 *   resampled_out 1 if the ensemble was resampled, else 0 (or NULL)
 * The library draws no random numbers: the resampling offset u and the
 * perturbations beta are the caller's (the tests and the benchmark take them
 * from numpy's PCG64 stream seeded with (seed, 0xF1, window), u first, then
 * beta_i = 1 + 0.05 N(0, 1) -- paper_2302_08341_gb300.synth.pf_draws), so a
 * C caller that wants the same particles must supply the same numbers.
 * Asynchronous (outputs valid after the stream is synchronised).
 * Errors: FLOOD_ERR_ARG (sizes, u outside [0,1)), FLOOD_ERR_STATE.
 */
int pf_assimilate(flood_grid* g, int n_gauges, const float* y, const double* d,
                  const double* sigma, double sigma_rel, double n_thr_frac, int force_resample,
                  double u, const float* beta, double* weights_out, int32_t* idx_out,
                  double* neff_out, int32_t* resampled_out, void* stream);

/*
 * pf_resample_systematic -- DA step (IV) alone: idx[j] = the particle whose
 * cumulative-weight interval [c_{i-1}, c_i) holds (u + j)/n, with the
 * cumulative sum taken in index order in FP64 and c_{n-1} set to 1.
 * w: [n] FP64, idx: [n] int32 (host or device).  Asynchronous.
 */
int pf_resample_systematic(int n, const double* w, double u, int32_t* idx, void* stream);

/* Observations of a gauge-misfit loss (adjoint, extension beyond the paper). */
typedef struct {
    int32_t n_samples;     /* observation times t0 + s * sample_dt, s = 1..n_samples      */
    int32_t n_gauges;
    double sample_dt;      /* seconds between observations (> 0)                         */
    const int32_t* cells;  /* [n_gauges] flat cell indices r * nx + c (host or device)    */
    const double* d;       /* [n_samples][n_gauges] observed depths (host or device)      */
} flood_loss_spec;

/*
 * flood_adjoint -- gradients by reverse mode (extension: the paper has no
 * adjoint).  All members must be at the same time t0.  The ensemble advances
 * through [t0, t0 + n_samples * sample_dt] exactly as flood_step would (it is
 * at the window's end afterwards), and for every member i the loss
 *     L_i = sum_s sum_k (h_i(t_s)[cells[k]] - d[s][k])^2
 * is differentiated with the step lengths held at the recorded schedule and
 * the derivative of the branch taken at every kink (Eq. 3's max, limiter,
 * wet/dry test, outflow clip, negative-depth clamp).  Memory: a checkpoint
 * every ckpt_every steps (0: about sqrt(steps)) plus ckpt_every + 1 replayed
 * states, each 12 bytes per cell per member.
 *   grad_n      [ny][nx] FP32  sum_i dL_i/dn_base (or NULL)
 *   grad_rain   [N] FP64       dL_i/d(rain multiplier of i) (or NULL)
 *   grad_scale  [N] FP64       dL_i/d(Manning scale of i) (or NULL)
 *   grad_h0     [N][ny][nx] FP32 dL_i/dh_i(t0) (or NULL)
 *   loss_out    [N] FP64       L_i (or NULL)
 * Synchronous.  Errors: FLOOD_ERR_ARG, FLOOD_ERR_STATE (members at different
 * times), FLOOD_ERR_OOM, FLOOD_ERR_NAN, FLOOD_ERR_TIMEOUT.
 */
int flood_adjoint(flood_grid* g, const flood_loss_spec* loss, int ckpt_every, float* grad_n,
                  double* grad_rain, double* grad_scale, float* grad_h0, double* loss_out,
                  void* stream);

/* Device time (ms, CUDA events) of the last flood_adjoint's forward pass
 * (with checkpointing) and of its reverse pass (replay included). */
int flood_adjoint_timing(const flood_grid* g, double* forward_ms, double* reverse_ms);

/* ==== Inflow hydrograph boundary ============================================
 * A discharge series Q (m^3/s, one value per rain block, FP32) entering the
 * domain through the west-edge links of rows [r0, r1), spread evenly: each
 * such link carries q = Q / (dx (r1 - r0)) into the domain instead of the
 * wall's zero (every member alike); the inflow volume is reported by
 * flood_inflow_volume and storage = rain + inflow - outflow + clamp
 * (- drained).  n_blocks = 0 removes the boundary.  Synchronous.
 * Errors: FLOOD_ERR_ARG (rows outside the grid, negative or non-finite
 * discharges).  flood_adjoint covers it: the inflow flux is prescribed, so it
 * has no derivative of its own, but it enters the depths (and the clamp
 * decisions) that every other derivative is taken at. */
int flood_set_inflow(flood_grid* g, int r0, int r1, const float* series, int n_blocks);
int flood_inflow_volume(flood_grid* g, double* volume);

/* ==== Streamflow gauges (the stream gauges of Section 4.1 / 4.4) ============
 * A section is a straight line of links: axis 0, the links east of cells
 * (r, fixed) for rows r in [start, end); axis 1, the links south of cells
 * (fixed, c) for columns c in [start, end).  Its discharge is
 * Q = sum of q dx over those links (m^3/s, positive toward increasing index);
 * fixed = nx - 1 (axis 0) or ny - 1 (axis 1) gives the outflow through an
 * edge.  Observed with a relative error (Section 4.4: sigma = 0.05 d), these
 * feed pf_assimilate as caller-supplied outputs y. */
typedef struct {
    int axis;       /* 0: x links, 1: y links */
    int fixed;      /* the column (axis 0) or row (axis 1) of the cells */
    int start, end; /* the rows (axis 0) or columns (axis 1), [start, end) */
} flood_section;

/* q_out [N][n_sections] FP32 (host or device): every member's discharge
 * through every section (FP64 sums).  Synchronous.  Errors: FLOOD_ERR_ARG
 * (a section outside the grid), FLOOD_ERR_STATE, FLOOD_ERR_OOM. */
int flood_flow_sample(flood_grid* g, int n_sections, const flood_section* sections,
                      float* q_out, void* stream);

/* ==== Land cover (Section 4.1, Table 1) =====================================
 * A class per cell (at most 4 classes), each with a Manning n (the members'
 * default; Table 1 gives 0.15 green land, 0.020 water bodies, 0.017
 * hardened ground), a runoff coefficient (the share of the rain that stays
 * on the surface: 0.9 on green land), a drainage flag (the pipe network's
 * drainage capacity I_drn applies: hardened ground) and an outside-the-
 * domain flag.  Per member: the Manning n of every class and the drainage
 * rate, the uncertain inputs of the paper's ensemble; a resampling carries
 * them with their particle.  Each step then uses, per cell,
 *   n = the member's n of the cell's class (times its Manning scale),
 *   h* = h + dt/dx (net inflow) + runoff(class) * rain depth,
 *   h' = h* - min(drains(class) * drainage rate * dt, max(h*, 0)),
 * and reports the drained volume (flood_drained_volume); storage = rain -
 * outflow + clamp - drained.  Cells outside the domain get their bed raised
 * to 1e6 m and no rain, so no link into them carries flow (Eq. 3); they are
 * held dry and at rest (flood_set_land_cover, flood_ensemble_init and
 * flood_set_state zero their depth and link fluxes), so the ordinary step of
 * the TMA engine launches only the tiles (128 columns x the strip height)
 * that hold a cell of the domain, with the same results as a step over
 * every tile.
 * flood_adjoint covers it: the Manning gradients are then taken with
 * respect to each member's own n at each cell (the class's), the rain
 * multiplier's gradient weighs each cell by its runoff coefficient, and a
 * cell that drainage emptied (h* > 0 and h' = 0) passes no sensitivity, like
 * a clamped one; the drainage rate's gradient comes from flood_adjoint_land_grad.
 * Not covered: a roughness factor field (refused either way).  Batches of
 * scenarios take land cover through flood_batch_set_land_cover. */
typedef struct {
    float n;        /* Manning n of the class (s m^-1/3), > 0 */
    float runoff;   /* share of the rain that stays on the surface, [0, 1] */
    int drains;     /* 1: the member's drainage rate applies to the class */
    int outside;    /* 1: cells of the class lie outside the domain */
} flood_land_class;

/* Set the land cover once per grid: cls [ny][nx] uint8 (< n_classes <= 4),
 * host or device.  Per-member parameters start at the classes' n and no
 * drainage (also after a later flood_ensemble_init).  Synchronous.
 * Errors: FLOOD_ERR_ARG, FLOOD_ERR_STATE (set twice, or a roughness factor
 * field is set), FLOOD_ERR_OOM. */
int flood_set_land_cover(flood_grid* g, const uint8_t* cls, int n_classes,
                         const flood_land_class* classes);

/* Per-member land-cover parameters: n_class [N][n_classes] (> 0) and
 * drain_rate [N] (m/s, >= 0), host or device; either may be NULL (kept).
 * Synchronous.  Errors: FLOOD_ERR_STATE (no land cover or ensemble),
 * FLOOD_ERR_ARG. */
int flood_set_land_params(flood_grid* g, const float* n_class, const float* drain_rate);
int flood_get_land_params(flood_grid* g, float* n_class, float* drain_rate);

/* Volume removed by drainage so far, per member [N] FP64 (m^3; zeros
 * without land cover).  Synchronous. */
int flood_drained_volume(flood_grid* g, double* drained);

/* Land-cover gradients of the last flood_adjoint, which must be the last
 * call to change the ensemble.  Host memory, either may be NULL:
 *   grad_n_class [N][n_classes] FP64  dL_i/dn_k: member i's per-cell Manning
 *                gradients summed over the cells of class k (FP64, a fixed
 *                order; needs an adjoint that was given grad_n)
 *   grad_drain   [N] FP64  dL_i/d(drainage rate of i): minus dt times the
 *                sensitivity to the depth after the step, summed over the
 *                steps and the cells of draining classes that drainage left
 *                wet (a cell it emptied passes nothing)
 * Synchronous.  Errors: FLOOD_ERR_STATE (no land cover, no fresh adjoint, or
 * grad_n_class after one without grad_n), FLOOD_ERR_OOM, FLOOD_ERR_CUDA. */
int flood_adjoint_land_grad(flood_grid* g, double* grad_n_class, double* grad_drain,
                            void* stream);

/* ==== Ensemble products (Section 4.4, Figs. 15-16) ==========================
 * Per member, the running maximum depth hmax_i(r, c) over every step since
 * tracking was turned on; from those and the particle weights w_i, per cell:
 *   exceedance  P = sum_i w_i [hmax_i >= threshold]   (the threshold rounded
 *               to FP32, result FP32)
 *   percentile  h_a = the smallest hmax_i whose weighted empirical
 *               distribution value W_i = sum of w_j over members j with
 *               hmax_j <= hmax_i reaches a; where every W_i stays below a,
 *               the largest hmax_i.
 * The sums are exact: each weight is rounded once to a whole number of
 * units of 2^-60 (to nearest, ties to even) and the units are added as
 * 64-bit integers, so no summation order changes a map; W_i reaches a when
 * W_i >= ceil(a 2^60) units, and P is the unit sum times 2^-60 rounded to
 * FP64, then to FP32.  Weights must lie in [0, 1] and sum to about one. */

/* Turn tracking on (1: the maxima start at the current depths) or off (0).
 * While on, every step also raises the maxima (8 more bytes per
 * member-cell-step), and a resampling copies a particle's maxima along with
 * its state.  Errors: FLOOD_ERR_STATE (before flood_ensemble_init),
 * FLOOD_ERR_OOM. */
int flood_track_max_depth(flood_grid* g, int on, void* stream);

/* Member m's running maximum depth as [ny][nx] FP32 (host or device).
 * Synchronous.  Errors: FLOOD_ERR_STATE (not tracking), FLOOD_ERR_ARG. */
int flood_get_max_depth(flood_grid* g, int member, float* out, void* stream);

/* The products above with the current particle weights.  exceed: [ny][nx]
 * FP32 or NULL; levels: n_levels (0..16) values in (0, 1]; pct:
 * [n_levels][ny][nx] FP32.  Host or device outputs.  One thread per cell
 * sorts the cell's maxima in registers (up to 128 members; with unequal
 * weights as 32-bit keys carrying the member index; more members are
 * staged in shared memory).  A percentile of a value that ties -0 with +0
 * may come out as either zero.  Maxima must not be NaN.  Synchronous.  Errors:
 * FLOOD_ERR_STATE (not tracking, or weights outside [0, 1] or summing far
 * above one), FLOOD_ERR_ARG (levels, more than 384 members or 65535 rows),
 * FLOOD_ERR_OOM. */
int flood_ensemble_products(flood_grid* g, double threshold, int n_levels, const double* levels,
                            float* exceed, float* pct, void* stream);

/* ==== Gradient calibration (extension: the paper estimates its uncertain
 * inputs with the particle filter alone, Section 2.2 / 4.4) ================
 * Roughness as the base field times a coarse factor field: fine cell (r, c)
 * lies in block (floor(r cy / ny), floor(c cx / nx)) and uses
 *     n(r, c) = n0(r, c) * f[block],
 * n0 the base field given to flood_create_grid.  The calibration step moves
 * the per-member rain multipliers and f along the gradients of the last
 * flood_adjoint. */

/* Set the factor field: f [cy][cx] FP32, host or device, every value > 0;
 * 1 <= cy <= ny, 1 <= cx <= nx.  Rewrites the roughness field on the device
 * (n0 is kept from the first call).  Synchronous.
 * Errors: FLOOD_ERR_ARG, FLOOD_ERR_STATE (land cover is set: the roughness
 * then comes from the classes), FLOOD_ERR_OOM, FLOOD_ERR_CUDA. */
int flood_set_roughness_factor(flood_grid* g, int cy, int cx, const float* f, void* stream);

/* The factor field in use: writes its shape and, if f is not NULL, its
 * values ([cy][cx] FP32, host or device).  Synchronous.
 * Errors: FLOOD_ERR_STATE if no factor field was set. */
int flood_get_roughness_factor(flood_grid* g, int* cy, int* cx, float* f);

/* Gradient of the last flood_adjoint's total loss L = sum_i L_i with respect
 * to the factor field: grad[b] = sum over the cells of block b of
 * n0 * dL/dn, in FP64 (a fixed-order reduction per block).  grad: [cy][cx]
 * FP64, host or device.  The adjoint must have been given grad_n and nothing
 * may have changed the ensemble since (a step, the particle filter, set
 * state / members / factor).  Synchronous.
 * Errors: FLOOD_ERR_STATE (no factor field, or no such adjoint). */
int flood_roughness_factor_grad(flood_grid* g, double* grad, void* stream);

/*
 * flood_calibration_step -- one descent step from the last flood_adjoint
 * (same precondition as flood_roughness_factor_grad; grad_n is only needed
 * when a factor field is set).  In log-parameter space with the Polyak step
 * of a loss whose minimum is zero, each component clipped to [-delta, delta]:
 *   member i:  m_i <- m_i exp(clip(-eta L_i / g_i)),  g_i = m_i dL_i/dm_i
 *   field:     f_b <- f_b exp(clip(-eta L G_b / |G|^2)),  G_b = f_b dL/df_b,
 *              L = sum_i L_i, then n = n0 * f
 *   land cover, member i: one joint step over all of its parameters,
 *              theta = (its rain multiplier, its n of every class, its
 *              drainage rate), in place of the member step above:
 *              theta_j <- theta_j exp(clip(-eta L_i G_j / |G|^2)),
 *              G_j = theta_j dL_i/dtheta_j (flood_adjoint_land_grad), so the
 *              step removes eta L_i to first order once; after an adjoint
 *              without grad_n the class roughness stays and the step runs
 *              over the rain multiplier and drainage rate
 * (g_i = 0 or |G| = 0 leaves the parameters unchanged).  L_i is recomputed on
 * the device from the adjoint's recorded gauge outputs.  loss_out [N] FP64
 * (host or device, or NULL) receives L_i.  After the step the adjoint is
 * spent: another step needs another flood_adjoint.  Synchronous.
 * Errors: FLOOD_ERR_ARG (eta <= 0, delta <= 0), FLOOD_ERR_STATE.
 */
int flood_calibration_step(flood_grid* g, double eta, double delta, double* loss_out,
                           void* stream);

/* Copy member m's state out / in: h, qx, qy as [ny][nx] FP32 in the link
 * convention above (any may be NULL).  Asynchronous. */
int flood_get_state(flood_grid* g, int member, float* h, float* qx, float* qy, void* stream);
int flood_set_state(flood_grid* g, int member, const float* h, const float* qx,
                    const float* qy, void* stream);

/* Per-member scalars, each [N] (any may be NULL): time (s), steps taken,
 * rain multiplier, Manning scale, particle weight, maximum depth.
 * Synchronous. */
int flood_get_members(flood_grid* g, double* t, int64_t* steps, float* rain_mult,
                      float* manning_scale, double* weights, float* hmax);

/* Set per-member rain multipliers, Manning scales or weights (NULL = keep).
 * Synchronous. */
int flood_set_members(flood_grid* g, const float* rain_mult, const float* manning_scale,
                      const double* weights);

/*
 * flood_volume_report -- FP64 volume bookkeeping per member (m^3), each [N]
 * (any may be NULL): current storage sum(h) dx^2, rain added, volume that
 * left through free-outflow edges, and volume added by clamping negative
 * depths to zero.  Conservation: storage(t) - storage(t0) = rain - outflow
 * + clamp up to FP32 rounding of the state.  Synchronous.
 */
int flood_volume_report(flood_grid* g, double* storage, double* rain, double* outflow,
                        double* clamp);

/* Number of kernels this grid has launched so far (for launch accounting). */
int64_t flood_launch_count(const flood_grid* g);

/* Per-launch timing of the step kernel with CUDA events recorded on the
 * launching stream around every step launch.  Synchronises the device, writes
 * the step-kernel time (ms) and launch count accumulated since the previous
 * call (either pointer may be NULL), resets them, and turns timing on
 * (enable = 1) or off (enable = 0). */
int flood_profile(flood_grid* g, int enable, double* step_kernel_ms, int64_t* step_launches);

/* Launch shape of the step kernel (for tuning): each warp marches down
 * rows_per_strip rows of a 128-column span of one member; a CTA holds
 * members_per_cta members (1, 2, 4 or 8) of the same span(s).  (0, 0) restores
 * the automatic choice.  Applies to the following steps; results do not depend
 * on it (bitwise).  Errors: FLOOD_ERR_ARG. */
int flood_set_launch(flood_grid* g, int rows_per_strip, int members_per_cta);
int flood_get_launch(const flood_grid* g, int* rows_per_strip, int* members_per_cta);

/* Step-kernel engine: 0 = direct float4 loads, 1 = rows staged through shared
 * memory by the tensor memory accelerator (default where available), 2 = the
 * plain form kept for comparison: one launch per member per step with direct
 * loads (the bed and roughness are then read once per member, not once per
 * tile of several members).  All give identical results.  Errors:
 * FLOOD_ERR_ARG. */
int flood_set_engine(flood_grid* g, int engine);

/* Failure-detection hook: the number of SM clock cycles each bounded wait of
 * the TMA step kernel for a staged row may take before the kernel gives up
 * (default 2e8, about 0.1 s; cycles < 0 restores it).  A kernel that gives
 * up first waits, with the default limit, for every copy it still has in
 * flight, records FLOOD_ERR_TIMEOUT in the grid's error word and returns; the
 * next synchronising call (flood_step with t_end, flood_sync, a state read)
 * reports FLOOD_ERR_TIMEOUT, and every later step is a no-op until
 * flood_ensemble_init clears the word.  0 reduces each wait to a single
 * non-blocking test, which gives up on a row whose copy is still in flight:
 * that is how the tests reach the path.  A changed budget applies to the
 * plain step (no running maximum, land cover or checkpoints; a step with
 * them returns FLOOD_ERR_STATE), which is compiled separately so that the
 * ordinary step keeps its limit as a constant.  Errors: FLOOD_ERR_ARG. */
int flood_set_wait_budget(flood_grid* g, int64_t cycles);

/* CUDA-graph replay of flood_step (extension; the paper launches its kernels
 * one by one).  With on != 0, flood_step captures a run of 24 steps (the plan
 * and step kernels of each, in order) once, on a stream of the grid's own, and
 * replays that graph on the caller's stream for every further run of 24 steps
 * while every launch argument stays the same: t_end, the engine and launch
 * shape, land cover, the running maximum, inflow and the device buffers.  A
 * change captures again.  The steps before the member-clock ring returns to
 * its first slot and the remainder launch one by one.  Results are bit for bit
 * those of plain launches.  Steps timed by flood_profile and the adjoint's
 * logged forward launch plainly.  Off by default.  Errors: FLOOD_ERR_ARG;
 * flood_step reports a failed capture as FLOOD_ERR_CUDA. */
int flood_set_graphs(flood_grid* g, int on);

/* How many runs flood_step has captured into a graph and how many it has
 * replayed (either pointer may be NULL).  Errors: FLOOD_ERR_ARG. */
int flood_graph_stats(flood_grid* g, int64_t* captures, int64_t* replays);

/* Autotuner: time every step-kernel configuration (engine x rows per strip
 * {32, 64, 128} x members per CTA {8, 4, 2, 1}; 8 and 2 with the plain TMA
 * step only) for steps_per_trial steps on the
 * live ensemble, keep the fastest, and restore the ensemble (state, clocks,
 * volume counters) to where it was.  Writes the choice and its time per step
 * (ms); any output may be NULL.  Synchronous. */
int flood_autotune(flood_grid* g, int steps_per_trial, int* best_rows, int* best_mpc,
                   int* best_engine, double* best_ms, void* stream);

/* Wait for `stream`, then report device-side faults of the method: returns
 * FLOOD_ERR_NAN if any step produced a non-finite depth. */
int flood_sync(flood_grid* g, void* stream);

/* ==== Uneven batches (extension beyond the paper) =========================
 * Many independent scenarios, each with its own grid size, bed, roughness,
 * storm, Manning scale and duration, advanced together: one launch per step
 * covers every scenario's tiles, each scenario with its own step length from
 * Eq. 4 on its own maximum depth; the launches are replayed from a CUDA graph
 * of a fixed number of steps.  Same scheme, arithmetic and results as a
 * single-member flood_grid of that scenario. */
typedef struct flood_batch flood_batch;

/* n scenarios: scenario i has ny[i] x nx[i] cells with bed z[i] and base
 * Manning n_base[i] ([ny[i]][nx[i]] FP32, host or device; copied).  One
 * flood_params for all.  Synchronous.  Errors: FLOOD_ERR_ARG, _OOM, _CUDA. */
int flood_batch_create(flood_batch** out, int n, const int32_t* ny, const int32_t* nx,
                       const float* const* z, const float* const* n_base, const flood_params* p);
int flood_batch_destroy(flood_batch* b);
const char* flood_batch_last_error(const flood_batch* b);

/* Start every scenario dry at t = 0: scenario i with hyetographs[i]
 * ([n_blocks[i]] rain rates per rain block, m/s), rain multiplier, Manning
 * scale, and its own end time t_end[i] (s).  Synchronous. */
int flood_batch_init(flood_batch* b, const float* const* hyetographs, const int32_t* n_blocks,
                     const float* rain_mult, const float* manning_scale, const double* t_end,
                     void* stream);

/* The same with n_members[i] >= 1 members per scenario (the members of a
 * scenario are an ensemble, Eq. 6-7: they share its bed, roughness, storm and
 * end time, and each has its own state, clock and step length (Eq. 4),
 * rain multiplier and Manning scale).  rain_mult and manning_scale hold one
 * value per member, scenario by scenario ([sum n_members]).  The warps that
 * step one tile of a scenario for its different members run next to one
 * another, so the tile's bed and roughness come from DRAM once for all of
 * them (Section 3.2's shared definitive data).  Members are indexed
 * scenario by scenario wherever per-member arrays are returned; with one
 * member per scenario this is flood_batch_init.  Synchronous.  Errors:
 * FLOOD_ERR_ARG (a count outside 1..4096, more than 2^20 members in all),
 * FLOOD_ERR_OOM. */
int flood_batch_init_members(flood_batch* b, const float* const* hyetographs,
                             const int32_t* n_blocks, const int32_t* n_members,
                             const float* rain_mult, const float* manning_scale,
                             const double* t_end, void* stream);

/* Advance every scenario to min(t_stop, t_end[i]) (a window end), each with
 * its own steps.  Synchronises `stream` between graph replays (engines 0-1)
 * or after the persistent launch (engine 2) to follow the scenarios' clocks.
 * Errors: FLOOD_ERR_STATE (before init, or no progress), FLOOD_ERR_NAN,
 * FLOOD_ERR_TIMEOUT. */
int flood_batch_step(flood_batch* b, double t_stop, void* stream);

/* Launch shape: rows per warp strip (1..4096) and warps per CTA (4 or 8);
 * results do not depend on it.  Synchronous. */
int flood_batch_set_launch(flood_batch* b, int rows_per_strip, int warps_per_cta);

/* Step-kernel engine of the batch: 0 = direct float4 loads, 1 = rows staged
 * through shared memory by the tensor memory accelerator, each scenario with
 * its own tensor maps (the default where available), replayed as CUDA graphs
 * of one plan and one step launch per step; 2 = the same TMA-staged march in
 * one persistent cooperative launch per flood_batch_step call, looping plan
 * phase -> grid barrier -> step phase (warps draw tasks from a counter) ->
 * grid barrier until every scenario has reached the stop.  The barrier waits
 * are bounded: one that runs out makes the call return FLOOD_ERR_TIMEOUT.
 * Identical results.  Synchronous.  Errors: FLOOD_ERR_ARG, FLOOD_ERR_STATE
 * (engines 1-2 without tensor maps, engine 2 without cooperative launch). */
int flood_batch_set_engine(flood_batch* b, int engine);

/* Failure-detection hook of the persistent batched form: the number of SM
 * clock cycles a CTA may wait at the grid barrier (default 2e8, about 0.1 s;
 * cycles < 0 restores it).  A wait that runs out records FLOOD_ERR_TIMEOUT in
 * the batch's error word and every CTA leaves at its next barrier (no copy is
 * in flight at a barrier); the flood_batch_step call returns FLOOD_ERR_TIMEOUT
 * and flood_batch_init clears the word.  0 makes a CTA that is not the last
 * to arrive give up at once.  Errors: FLOOD_ERR_ARG. */
int flood_batch_set_wait_budget(flood_batch* b, int64_t cycles);

/* Scenario i's state (its first member) as [ny[i]][nx[i]] FP32 arrays (any
 * may be NULL). */
int flood_batch_get_state(flood_batch* b, int i, float* h, float* qx, float* qy, void* stream);
/* The state of member m of scenario i. */
int flood_batch_get_member_state(flood_batch* b, int i, int m, float* h, float* qx, float* qy,
                                 void* stream);

/* Per-member clocks and FP64 volumes, each [sum of the members], scenario by
 * scenario ([n] with one member per scenario; any may be NULL).
 * Synchronous. */
int flood_batch_members(flood_batch* b, double* t, int64_t* steps, double* storage, double* rain,
                        double* outflow, double* clamp);

/* Step kernels launched so far (graph replays count every launch). */
int64_t flood_batch_launch_count(const flood_batch* b);

/* Autotuner of the batched step: time every configuration (rows per strip
 * {16, 32, 64} x warps per CTA {4, 8} with the graph-replayed TMA engine, and
 * {16, 32, 64} x 4 warps with the persistent engine where the device has
 * cooperative launch; direct loads without tensor maps) on the live batch,
 * each advancing every scenario trial_s seconds past the latest current time
 * (after an untimed run of the same trial), keep the fastest, and put the
 * batch back exactly as it was (states, clocks, rain and volume sums).
 * Writes the choice and its trial time (ms); any output may be NULL.
 * Synchronous.  Errors: FLOOD_ERR_ARG (trial_s <= 0), FLOOD_ERR_STATE (before
 * flood_batch_init), FLOOD_ERR_OOM (the state snapshot), and those of
 * flood_batch_step. */
int flood_batch_autotune(flood_batch* b, double trial_s, int* best_rows, int* best_warps,
                         int* best_engine, double* best_ms, void* stream);

/* Land cover of scenario `scen` (Section 4.1; the same classes, rules and
 * arithmetic as flood_set_land_cover on a grid): cls [ny][nx] uint8
 * (< n_classes <= 4), host or device.  Set before flood_batch_init, for
 * every scenario of the batch or for none (flood_batch_init refuses a mix).
 * The bed of cells outside the domain is raised out of reach and they get
 * no rain; the tiles (128 columns x the strip height) that hold no cell of
 * the domain are not scheduled.  Each member starts with the classes' n and
 * no drainage at every flood_batch_init.  Synchronous.  Errors:
 * FLOOD_ERR_ARG, FLOOD_ERR_STATE (after flood_batch_init, or set twice),
 * FLOOD_ERR_OOM. */
int flood_batch_set_land_cover(flood_batch* b, int scen, const uint8_t* cls, int n_classes,
                               const flood_land_class* classes);

/* Land-cover parameters of the members of scenario `scen`: n_class
 * [members][n_classes] (> 0) and drain_rate [members] (m/s, >= 0), host or
 * device; either may be NULL (kept).  Synchronous.  Errors: FLOOD_ERR_STATE
 * (no land cover, or before flood_batch_init), FLOOD_ERR_ARG. */
int flood_batch_set_land_params(flood_batch* b, int scen, const float* n_class,
                                const float* drain_rate);

/* Volume removed by drainage so far, per member [sum of the members] FP64
 * (m^3; zeros without land cover); storage = rain - outflow + clamp -
 * drained.  Synchronous. */
int flood_batch_drained_volume(flood_batch* b, double* drained);

/* ==== Allocation-free volume reduction ======================================
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- code running inside a stream capture, under a
 * device-memory budget owned by an embedding application, or in a real-time
 * loop that must never wait on the allocator. */

/* Largest number of rows flood_storage_static accepts (its block partials
 * live in a fixed device array of FLOOD_STATIC_MAX_ROWS / 16 doubles, 32 KB,
 * held by every device that loads the library until the process exits). */
#define FLOOD_STATIC_MAX_ROWS 65536

/*
 * flood_storage_static -- *out = dx^2 * sum of h over a depth field, in FP64,
 * without allocating anything.
 *   h    device pointer to ny rows of ld floats (only the first nx of each row
 *        are summed); the caller owns it
 *   out  device pointer to one double; the caller owns it
 * Same arithmetic and order as the storage reported by flood_volume_report,
 * so the two agree bit for bit on the same field.  Asynchronous on `stream`.
 * The first call on a device (with that device current) looks up the device
 * address of the library's partials array; make that first call before any
 * stream capture.  Every call on a device shares that array and overwrites
 * the part it uses: calls that can overlap on the GPU (unordered streams)
 * race and must be serialised by the caller.
 * Errors: FLOOD_ERR_ARG (NULL pointer, ny > FLOOD_STATIC_MAX_ROWS, ld < nx,
 * dx <= 0), FLOOD_ERR_CUDA; message from flood_storage_static_error().
 */
int flood_storage_static(const float* h, int ny, int nx, int ld, double dx, double* out,
                         void* stream);
const char* flood_storage_static_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FLOOD_H */
