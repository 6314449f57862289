/*
 * FP64 CPU oracle for the ensemble local-inertial flood model and its
 * particle filter (Wei et al., "Enable high-resolution, real-time ensemble
 * simulation and data assimilation of flood inundation using distributed GPU
 * parallelization", arXiv 2302.08341).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Layout (the paper's link picture, Section 3.1, Fig. 2):
 *   cells   h[r][c], z[r][c], n[r][c]            r = 0..ny-1, c = 0..nx-1
 *   x links qx[r][c]  c = 0..nx   link between cell (r,c-1) and (r,c);
 *                     c = 0 is the west edge, c = nx the east edge
 *   y links qy[r][c]  r = 0..ny   link between cell (r-1,c) and (r,c);
 *                     r = 0 is the north edge, r = ny the south edge
 * q is flow per unit width (m^2/s), positive toward increasing index.
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes): x runs along columns and y along rows; Eq. 1 is read as
 * dh = dt * dV / (dx dy) with dV the net volume flux of Eq. 5; the surface
 * slope in Eq. 2 is (eta_2 - eta_1)/dx along +axis; a link carries no flow
 * when its flow depth (Eq. 3) is zero (or below an optional threshold h_eps,
 * default 0); each link is limited to a quarter of the upstream
 * cell's volume per step; free-outflow edges use a ghost cell one edge slope
 * lower with the edge cell's depth (normal-depth boundary) and pass outward
 * flow only; the west and north edges are walls.
 *
 * Parity pins: every function here is checked by the CPU tests against
 * closed forms, invariants or the paper's printed numbers (time-step pin of
 * Section 4.1, Manning normal flow, seiche period sqrt(g h), lake at rest,
 * uniform rain, exact volume balance, x/y transposition symmetry; scipy's
 * Gaussian density for Eq. 9-11, brute-force enumeration of systematic
 * resampling; Eq. 4 at a known maximum depth through the evolution loop, a
 * gauge sample of a field whose values name their member and cell, the
 * ensemble loop equal to each member evolved alone).  No function is left
 * without a pin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ny, nx;
    double dx;            /* cell size, dx = dy (m)                          */
    double g;             /* gravitational acceleration (m s^-2)             */
    double alpha;         /* Courant coefficient k of Eq. 4                  */
    double dt_cap;        /* upper bound on the time step (s)                */
    double dt_fixed;      /* > 0: use this fixed step instead of Eq. 4       */
    double h_eps;         /* links with flow depth <= h_eps carry no flow (m);
                             0 = Eq. 2-3 as printed: no flow only when the
                             flow depth is zero                              */
    double h_floor;       /* floor on h_max inside Eq. 4 (m)                 */
    double rain_block;    /* length of one piecewise-constant rain block (s) */
    double edge_slope;    /* bed slope that places the outflow ghost cell    */
    int limiter;          /* 1: |q| <= h_upstream dx / (4 dt) on each link   */
    int east_outflow;     /* 1: free outflow through the east edge           */
    int south_outflow;    /* 1: free outflow through the south edge          */
    /* Land cover (Section 4.1), both NULL when absent: per cell, the fraction
       of the rain that stays on the surface (the runoff coefficient) and the
       drainage rate (m/s) that removes water while there is any. */
    const double* rc;
    const double* drain;
    /* Inflow hydrograph (NULL when absent): a discharge series (m^3/s, one
       value per rain block) entering through the west edge links of rows
       [inflow_r0, inflow_r1), spread evenly over them; inflow_q is the flux
       per unit width (m^2/s) of the current step, set by orc_advance. */
    const double* inflow;
    int inflow_blocks, inflow_r0, inflow_r1;
    double inflow_q;
} orc_params;

/* Volume bookkeeping of one member (m^3), all in FP64. */
typedef struct {
    double rain;     /* rain volume added                                     */
    double outflow;  /* volume that left through free-outflow edges           */
    double clamp;    /* volume added by resetting negative depths to zero     */
    double drained;  /* volume removed by drainage (land cover)               */
    double inflow;   /* volume that entered through an inflow boundary         */
} orc_volumes;

#define IX(r, c) ((size_t)(r) * (size_t)nx + (size_t)(c))
#define IQX(r, c) ((size_t)(r) * (size_t)(nx + 1) + (size_t)(c))
#define IQY(r, c) ((size_t)(r) * (size_t)nx + (size_t)(c))

/* ---- Eq. 4: time step ---------------------------------------------------
 * dt_max = k dx / sqrt(g h_max), with h_max floored at h_floor and the step
 * capped at dt_cap (or a fixed step), then shortened so the member lands
 * exactly on the next stop: the end of the current rain block (rain is
 * re-assigned every block, step (I) of Section 3.1) or t_end if that comes
 * first (t_end < 0: no end).  Returns dt and writes the time after the step. */
double orc_dt(const orc_params* p, double hmax, double t, double t_end, double* t_next)
{
    double dt;
    if (p->dt_fixed > 0.0) {
        dt = p->dt_fixed;
    } else {
        double hm = hmax > p->h_floor ? hmax : p->h_floor;
        dt = p->alpha * p->dx / sqrt(p->g * hm);
        if (dt > p->dt_cap) dt = p->dt_cap;
    }
    double stop = (floor(t / p->rain_block) + 1.0) * p->rain_block;
    if (t_end >= 0.0 && t_end < stop) stop = t_end;
    if (t + dt >= stop) {
        dt = stop - t;
        *t_next = stop;
    } else {
        *t_next = t + dt;
    }
    return dt;
}

/* Rain rate (m/s) of the block holding time t: step (I) of Section 3.1. */
double orc_rain_rate(const orc_params* p, const double* hyeto, int n_blocks, double t)
{
    double b = floor(t / p->rain_block);
    if (b < 0.0 || b >= (double)n_blocks) return 0.0;
    return hyeto[(int)b];
}

/* ---- Eq. 3 and Eq. 2: flux on one link -----------------------------------
 * Cell 1 is on the low-index side, cell 2 on the high-index side; q > 0 flows
 * from 1 to 2.  nl is the link's Manning coefficient. */
double orc_link_flux(const orc_params* p, double h1, double z1, double h2, double z2,
                     double q, double nl, double dt)
{
    double eta1 = h1 + z1, eta2 = h2 + z2;
    double hflow = fmax(eta1, eta2) - fmax(z1, z2);                 /* Eq. 3 */
    if (hflow <= p->h_eps) return 0.0;
    double S = (eta2 - eta1) / p->dx;                  /* water-surface slope */
    double num = q - p->g * hflow * dt * S;
    /* friction term g n^2 |q_t| dt / h_flow^(7/3); exactly 0 when q_t = 0.
       |q_t| multiplies h_flow^(-7/3) first, so that a vanishing flow depth
       (a wetting front's denormal depths) gives infinite friction, i.e. no
       flow, instead of 0/0 from two underflows. */
    double fric = q == 0.0 ? 0.0 : p->g * nl * nl * dt * (fabs(q) * pow(hflow, -7.0 / 3.0));
    double den = 1.0 + fric;
    double qn = num / den;                                          /* Eq. 2 */
    if (p->limiter) {
        double lim = (qn > 0.0 ? h1 : h2) * p->dx / (4.0 * dt);
        if (qn > lim) qn = lim;
        if (qn < -lim) qn = -lim;
    }
    return qn;
}

/* Free-outflow link from edge cell (h, z) into a ghost cell that continues
 * the bed at the edge slope and carries the same depth (zero depth gradient,
 * i.e. a normal-depth boundary); only outward (positive) flow passes. */
static double outflow_flux(const orc_params* p, double h, double z, double q, double nl, double dt)
{
    double qn = orc_link_flux(p, h, z, h, z - p->edge_slope * p->dx, q, nl, dt);
    return qn > 0.0 ? qn : 0.0;
}

/* ---- One numerical iteration of one member (steps III and IV) -------------
 * Fluxes on every link from the state at time t (Eq. 2-3), then the volume
 * change of every cell (Eq. 5) turned into depth (Eq. 1) with the rain of the
 * current block.  h, qx, qy are updated in place; qx_new/qy_new are scratch of
 * the link arrays' sizes.  scale multiplies the Manning field of this member;
 * rain is the member's rain rate (m/s) for this step. */
void orc_step(const orc_params* p, const double* z, const double* n, double scale,
              double rain, double dt, double* h, double* qx, double* qy,
              double* qx_new, double* qy_new, orc_volumes* vol)
{
    const int ny = p->ny, nx = p->nx;
    const double dx = p->dx;

    /* step (III): x links */
    for (int r = 0; r < ny; ++r) {
        for (int c = 0; c <= nx; ++c) {
            double qn;
            if (c == 0) {
                qn = (p->inflow && r >= p->inflow_r0 && r < p->inflow_r1)
                         ? p->inflow_q                                 /* inflow */
                         : 0.0;                                        /* west wall */
            } else if (c == nx) {
                qn = p->east_outflow
                         ? outflow_flux(p, h[IX(r, nx - 1)], z[IX(r, nx - 1)], qx[IQX(r, nx)],
                                        scale * n[IX(r, nx - 1)], dt)
                         : 0.0;
            } else {
                double nl = scale * 0.5 * (n[IX(r, c - 1)] + n[IX(r, c)]);
                qn = orc_link_flux(p, h[IX(r, c - 1)], z[IX(r, c - 1)], h[IX(r, c)], z[IX(r, c)],
                                   qx[IQX(r, c)], nl, dt);
            }
            qx_new[IQX(r, c)] = qn;
        }
    }
    /* step (III): y links */
    for (int r = 0; r <= ny; ++r) {
        for (int c = 0; c < nx; ++c) {
            double qn;
            if (r == 0) {
                qn = 0.0;                                         /* north wall */
            } else if (r == ny) {
                qn = p->south_outflow
                         ? outflow_flux(p, h[IX(ny - 1, c)], z[IX(ny - 1, c)], qy[IQY(ny, c)],
                                        scale * n[IX(ny - 1, c)], dt)
                         : 0.0;
            } else {
                double nl = scale * 0.5 * (n[IX(r - 1, c)] + n[IX(r, c)]);
                qn = orc_link_flux(p, h[IX(r - 1, c)], z[IX(r - 1, c)], h[IX(r, c)], z[IX(r, c)],
                                   qy[IQY(r, c)], nl, dt);
            }
            qy_new[IQY(r, c)] = qn;
        }
    }
    /* step (IV): volume change (Eq. 5) and depth (Eq. 1) of every cell */
    for (int r = 0; r < ny; ++r) {
        for (int c = 0; c < nx; ++c) {
            double dV = qx_new[IQX(r, c)] * dx - qx_new[IQX(r, c + 1)] * dx
                      + qy_new[IQY(r, c)] * dx - qy_new[IQY(r + 1, c)] * dx;     /* Eq. 5 */
            const double rcv = p->rc ? p->rc[IX(r, c)] : 1.0;
            double hn = h[IX(r, c)] + dt * dV / (dx * dx) + dt * rain * rcv;     /* Eq. 1 */
            if (p->drain) {
                /* drainage takes at most the water present after this step's
                   fluxes and rain */
                double sink = dt * p->drain[IX(r, c)];
                const double avail = hn > 0.0 ? hn : 0.0;
                if (sink > avail) sink = avail;
                hn -= sink;
                vol->drained += sink * dx * dx;
            }
            if (hn < 0.0) {
                vol->clamp += -hn * dx * dx;
                hn = 0.0;
            }
            h[IX(r, c)] = hn;
        }
    }
    for (int r = 0; r < ny; ++r) vol->outflow += dt * qx_new[IQX(r, nx)] * dx;
    for (int r = 0; r < ny; ++r) vol->inflow += dt * qx_new[IQX(r, 0)] * dx;
    for (int c = 0; c < nx; ++c) vol->outflow += dt * qy_new[IQY(ny, c)] * dx;
    if (p->rc) {
        double area = 0.0;
        for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) area += p->rc[i];
        vol->rain += dt * rain * dx * dx * area;
    } else {
        vol->rain += dt * rain * dx * dx * (double)ny * (double)nx;
    }
    memcpy(qx, qx_new, sizeof(double) * (size_t)ny * (size_t)(nx + 1));
    memcpy(qy, qy_new, sizeof(double) * (size_t)(ny + 1) * (size_t)nx);
}

double orc_hmax(int ny, int nx, const double* h)
{
    double m = 0.0;
    for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) m = h[i] > m ? h[i] : m;
    return m;
}

double orc_storage(int ny, int nx, double dx, const double* h)
{
    double v = 0.0;
    for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) v += h[i] * dx * dx;
    return v;
}

/* ---- Eq. 6: evolve one member until t_end -------------------------------
 * Repeats (dt by Eq. 4, rain of the block, one iteration) until the member's
 * time reaches t_end, or for max_steps steps (max_steps < 0: no limit).
 * If dt_log is non-NULL the dt of each step is written there (up to
 * dt_log_cap entries).  Returns the number of steps taken. */
long orc_advance(const orc_params* p, const double* z, const double* n, double scale,
                 double rain_mult, const double* hyeto, int n_blocks,
                 double* h, double* qx, double* qy, double* t, double t_end, long max_steps,
                 orc_volumes* vol, double* dt_log, long dt_log_cap)
{
    const int ny = p->ny, nx = p->nx;
    double* qx_new = (double*)malloc(sizeof(double) * (size_t)ny * (size_t)(nx + 1));
    double* qy_new = (double*)malloc(sizeof(double) * (size_t)(ny + 1) * (size_t)nx);
    long steps = 0;
    while ((t_end < 0.0 || *t < t_end) && (max_steps < 0 || steps < max_steps)) {
        double t_next;
        double dt = orc_dt(p, orc_hmax(ny, nx, h), *t, t_end, &t_next);
        double rain = orc_rain_rate(p, hyeto, n_blocks, *t) * rain_mult;
        orc_params ps = *p;
        if (p->inflow)
            ps.inflow_q = orc_rain_rate(p, p->inflow, p->inflow_blocks, *t) /
                          (p->dx * (double)(p->inflow_r1 - p->inflow_r0));
        orc_step(&ps, z, n, scale, rain, dt, h, qx, qy, qx_new, qy_new, vol);
        if (dt_log && steps < dt_log_cap) dt_log[steps] = dt;
        *t = t_next;
        ++steps;
    }
    free(qx_new);
    free(qy_new);
    return steps;
}

/* The same evolution for every member of an ensemble (members are
 * independent, Eq. 6), optionally spread over OpenMP threads.  State arrays
 * are member-major: h[M][ny][nx], qx[M][ny][nx+1], qy[M][ny+1][nx]. */
void orc_advance_ensemble(const orc_params* p, int M, const double* z, const double* n,
                          const double* scale, const double* rain_mult, const double* hyeto,
                          int n_blocks, double* h, double* qx, double* qy, double* t,
                          double t_end, long max_steps, orc_volumes* vol, long* steps, int nthreads)
{
    const size_t nc = (size_t)p->ny * (size_t)p->nx;
    const size_t nqx = (size_t)p->ny * (size_t)(p->nx + 1);
    const size_t nqy = (size_t)(p->ny + 1) * (size_t)p->nx;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int m = 0; m < M; ++m) {
        steps[m] = orc_advance(p, z, n, scale[m], rain_mult[m], hyeto, n_blocks, h + m * nc,
                               qx + m * nqx, qy + m * nqy, &t[m], t_end, max_steps, &vol[m],
                               NULL, 0);
    }
    (void)nthreads;
}

/* ---- DA step (I): model outputs at the gauges ----------------------------
 * y[m][g] = depth of member m at flat cell index cells[g]. */
void orc_gauge_sample(int M, int ncell, int G, const int32_t* cells, const double* h, double* y)
{
    for (int m = 0; m < M; ++m)
        for (int g = 0; g < G; ++g) y[(size_t)m * G + g] = h[(size_t)m * ncell + cells[g]];
}

/* ---- DA steps (II)-(III): Eq. 9-12 ----------------------------------------
 * Gaussian likelihood with diagonal covariance (Eq. 9), posterior weight
 * proportional to likelihood times prior weight (Eq. 10), normalisation
 * (Eq. 11) and the effective sample size (Eq. 12).  The constant
 * 1/sqrt((2 pi)^Nd |Sigma|) is common to all particles and cancels in
 * Eq. 11.  Products of small numbers are formed as sums of logarithms and
 * normalised by the largest term (log-sum-exp), which is Eq. 10-11 without
 * underflow.  sigma_rel > 0 selects Sigma = diag((sigma_rel d_g)^2), the
 * paper's relative error (Section 4.4); otherwise sigma[g] is used.
 * Returns 0, or -1 if every posterior weight is zero. */
int orc_pf_weights(int M, int G, const double* y, const double* d, const double* sigma,
                   double sigma_rel, const double* w_prior, double* w_post, double* neff)
{
    double* lw = (double*)malloc(sizeof(double) * (size_t)M);
    double lmax = -INFINITY;
    for (int i = 0; i < M; ++i) {
        double chi2 = 0.0;
        for (int g = 0; g < G; ++g) {
            double s = sigma_rel > 0.0 ? sigma_rel * d[g] : sigma[g];
            double e = (y[(size_t)i * G + g] - d[g]) / s;
            chi2 += e * e;
        }
        lw[i] = log(w_prior[i]) - 0.5 * chi2;           /* log of Eq. 10 */
        if (lw[i] > lmax) lmax = lw[i];
    }
    if (!(lmax > -INFINITY)) {
        free(lw);
        return -1;
    }
    double sum = 0.0;
    for (int i = 0; i < M; ++i) sum += exp(lw[i] - lmax);
    double s2 = 0.0;
    for (int i = 0; i < M; ++i) {
        w_post[i] = exp(lw[i] - lmax) / sum;                         /* Eq. 11 */
        s2 += w_post[i] * w_post[i];
    }
    *neff = 1.0 / s2;                                                /* Eq. 12 */
    free(lw);
    return 0;
}

/* ---- DA step (IV): systematic resampling -----------------------------------
 * Arulampalam et al. (2002), cited in Section 2.2: cumulative weights c_i
 * summed in index order (c_{M-1} set to 1), offsets u_j = (u + j)/M for one
 * uniform draw u in [0,1), idx[j] = the smallest i with c_i > u_j, i.e.
 * particle i owns the half-open interval [c_{i-1}, c_i) so a particle of zero
 * weight is never drawn (the tutorial's c_i >= u_j differs only when u_j
 * falls exactly on a cumulative weight). */
void orc_resample_systematic(int M, const double* w, double u, int32_t* idx)
{
    double* c = (double*)malloc(sizeof(double) * (size_t)M);
    double acc = 0.0;
    for (int i = 0; i < M; ++i) {
        acc += w[i];
        c[i] = acc;
    }
    c[M - 1] = 1.0;
    int i = 0;
    for (int j = 0; j < M; ++j) {
        double uj = (u + (double)j) / (double)M;
        while (i < M - 1 && c[i] <= uj) ++i;
        idx[j] = i;
    }
    free(c);
}

/* ---- DA step (V): which slot receives which particle ---------------------
 * From the resampled indices, particle i has k_i duplicates.  Survivors
 * (k_i >= 1) keep their own slot; the k_i - 1 extra copies of each particle,
 * taken in increasing particle order, fill the slots of the particles that
 * were dropped (k_i = 0), in increasing slot order.  src[s] is the particle
 * that slot s holds afterwards. */
void orc_assign_slots(int M, const int32_t* idx, int32_t* src)
{
    int* k = (int*)calloc((size_t)M, sizeof(int));
    for (int j = 0; j < M; ++j) k[idx[j]]++;
    int next_src = 0;
    for (int s = 0; s < M; ++s) {
        if (k[s] >= 1) {
            src[s] = s;
        } else {
            while (k[next_src] <= 1) ++next_src;
            src[s] = next_src;
            k[next_src]--;
        }
    }
    free(k);
}

/* ==== Adjoint (reverse mode) of one iteration ================================
 * Extension beyond the paper: gradients of a gauge-misfit loss with respect
 * to the Manning field, the member's rain multiplier and the initial depth.
 * The step lengths are held fixed (the recorded schedule); at the kinks of
 * Eq. 3 (max), the limiter, the wet/dry test, the outflow clip and the
 * negative-depth clamp the derivative of the branch actually taken is used,
 * ties in Eq. 3's max going to the first argument. */

/* Forward link flux with the partial derivatives of q' with respect to h1,
 * h2, the old flux q and the link roughness nl. */
static double link_flux_d(const orc_params* p, double h1, double z1, double h2, double z2,
                          double q, double nl, double dt, double* d_h1, double* d_h2,
                          double* d_q, double* d_nl)
{
    *d_h1 = *d_h2 = *d_q = *d_nl = 0.0;
    double eta1 = h1 + z1, eta2 = h2 + z2;
    double hflow = fmax(eta1, eta2) - fmax(z1, z2);                 /* Eq. 3 */
    if (hflow <= p->h_eps) return 0.0;
    int first = eta1 >= eta2;            /* which argument of max(eta1, eta2) */
    double S = (eta2 - eta1) / p->dx;
    double num = q - p->g * hflow * dt * S;
    double fric = q == 0.0 ? 0.0 : p->g * nl * nl * dt * (fabs(q) * pow(hflow, -7.0 / 3.0));
    double den = 1.0 + fric;
    double qn = num / den;                                          /* Eq. 2 */
    if (p->limiter) {
        double lim = (qn > 0.0 ? h1 : h2) * p->dx / (4.0 * dt);
        if (qn > lim) {
            *d_h1 = p->dx / (4.0 * dt);
            return lim;
        }
        if (qn < -lim) {
            *d_h2 = -p->dx / (4.0 * dt);
            return -lim;
        }
    }
    /* q' = num / den */
    double dq_dnum = 1.0 / den, dq_dfric = -qn / den;
    double dnum_dhf = -p->g * dt * S, dnum_dS = -p->g * hflow * dt;
    double dfric_dq = q == 0.0 ? 0.0 : fric / q;
    double dfric_dhf = -(7.0 / 3.0) * fric / hflow;
    double dfric_dnl = nl == 0.0 ? 0.0 : 2.0 * fric / nl;
    double dq_dhf = dq_dnum * dnum_dhf + dq_dfric * dfric_dhf;
    double dq_dS = dq_dnum * dnum_dS;
    *d_h1 = (first ? dq_dhf : 0.0) - dq_dS / p->dx;
    *d_h2 = (first ? 0.0 : dq_dhf) + dq_dS / p->dx;
    *d_q = dq_dnum + dq_dfric * dfric_dq;
    *d_nl = dq_dfric * dfric_dnl;
    return qn;
}

/* Reverse of orc_step.  State (h, qx, qy) is the input of the forward step;
 * (lh, lqx, lqy) hold the loss's sensitivities to the step's outputs on entry
 * and to its inputs on exit.  grad_n (per cell) accumulates dL/dn_base,
 * *grad_rain dL/d(rain multiplier) given the block rate, *grad_scale
 * dL/d(Manning scale), and *grad_drain (if not NULL; land cover)
 * dL/d(kappa) for the drainage field scaled by kappa, at kappa = 1. */
void orc_step_adjoint(const orc_params* p, const double* z, const double* n, double scale,
                      double rate, double rain_mult, double dt, const double* h, const double* qx,
                      const double* qy, double* lh, double* lqx, double* lqy, double* grad_n,
                      double* grad_rain, double* grad_scale, double* grad_drain)
{
    const int ny = p->ny, nx = p->nx;
    const double dx = p->dx, T = dt / dx;
    const size_t nqx = (size_t)ny * (size_t)(nx + 1), nqy = (size_t)(ny + 1) * (size_t)nx;
    double* qxn = (double*)calloc(nqx, sizeof(double));
    double* qyn = (double*)calloc(nqy, sizeof(double));
    double* dx1 = (double*)calloc(nqx * 4, sizeof(double));   /* d/dh1, d/dh2, d/dq, d/dnl */
    double* dy1 = (double*)calloc(nqy * 4, sizeof(double));
    double* lt = (double*)calloc((size_t)ny * nx, sizeof(double));
    /* recompute the forward links with their derivatives; an inflow link on
       the west edge is prescribed (no derivative) but enters the depth that
       decides the clamp */
    if (p->inflow)
        for (int r = p->inflow_r0; r < p->inflow_r1; ++r) qxn[IQX(r, 0)] = p->inflow_q;
    for (int r = 0; r < ny; ++r)
        for (int c = 1; c <= nx; ++c) {
            double* dd = dx1 + IQX(r, c) * 4;
            if (c == nx) {
                if (!p->east_outflow) continue;
                double hh = h[IX(r, nx - 1)], zz = z[IX(r, nx - 1)];
                double nl = scale * n[IX(r, nx - 1)];
                double a, b;
                double qn = link_flux_d(p, hh, zz, hh, zz - p->edge_slope * dx, qx[IQX(r, nx)], nl,
                                        dt, &a, &b, &dd[2], &dd[3]);
                if (qn > 0.0) {
                    dd[0] = a + b;   /* the ghost carries the edge depth */
                    qxn[IQX(r, c)] = qn;
                } else {
                    dd[2] = dd[3] = 0.0;
                }
                continue;
            }
            double nl = scale * 0.5 * (n[IX(r, c - 1)] + n[IX(r, c)]);
            qxn[IQX(r, c)] = link_flux_d(p, h[IX(r, c - 1)], z[IX(r, c - 1)], h[IX(r, c)],
                                         z[IX(r, c)], qx[IQX(r, c)], nl, dt, &dd[0], &dd[1], &dd[2],
                                         &dd[3]);
        }
    for (int r = 1; r <= ny; ++r)
        for (int c = 0; c < nx; ++c) {
            double* dd = dy1 + IQY(r, c) * 4;
            if (r == ny) {
                if (!p->south_outflow) continue;
                double hh = h[IX(ny - 1, c)], zz = z[IX(ny - 1, c)];
                double nl = scale * n[IX(ny - 1, c)];
                double a, b;
                double qn = link_flux_d(p, hh, zz, hh, zz - p->edge_slope * dx, qy[IQY(ny, c)], nl,
                                        dt, &a, &b, &dd[2], &dd[3]);
                if (qn > 0.0) {
                    dd[0] = a + b;
                    qyn[IQY(r, c)] = qn;
                } else {
                    dd[2] = dd[3] = 0.0;
                }
                continue;
            }
            double nl = scale * 0.5 * (n[IX(r - 1, c)] + n[IX(r, c)]);
            qyn[IQY(r, c)] = link_flux_d(p, h[IX(r - 1, c)], z[IX(r - 1, c)], h[IX(r, c)],
                                         z[IX(r, c)], qy[IQY(r, c)], nl, dt, &dd[0], &dd[1], &dd[2],
                                         &dd[3]);
        }
    /* continuity: the clamp passes no sensitivity, nor does drainage that
       takes all the water present (land cover: the depth left is then 0
       whatever the depth before it); the rain that stays is runoff x rain;
       drainage that leaves water behind removes dt x drain, all of it
       sensitive to the drainage rate */
    double gr = 0.0, gk = 0.0;
    for (int r = 0; r < ny; ++r)
        for (int c = 0; c < nx; ++c) {
            const double rcv = p->rc ? p->rc[IX(r, c)] : 1.0;
            double hpre = h[IX(r, c)] + T * (qxn[IQX(r, c)] - qxn[IQX(r, c + 1)] + qyn[IQY(r, c)] -
                                             qyn[IQY(r + 1, c)]) + dt * rate * rain_mult * rcv;
            int pass = hpre >= 0.0;
            if (p->drain && hpre > 0.0 && hpre <= dt * p->drain[IX(r, c)]) pass = 0;
            lt[IX(r, c)] = pass ? lh[IX(r, c)] : 0.0;
            gr += lt[IX(r, c)] * dt * rate * rcv;
            if (p->drain && hpre > dt * p->drain[IX(r, c)])
                gk -= lt[IX(r, c)] * dt * p->drain[IX(r, c)];
        }
    *grad_rain += gr;
    if (grad_drain) *grad_drain += gk;
    /* sensitivity to each new link flux, then back through Eq. 2-3 */
    double* lh_new = (double*)calloc((size_t)ny * nx, sizeof(double));
    for (size_t i = 0; i < (size_t)ny * nx; ++i) lh_new[i] = lt[i];
    for (int r = 0; r < ny; ++r)
        for (int c = 1; c <= nx; ++c) {
            const double* dd = dx1 + IQX(r, c) * 4;
            double mu = lqx[IQX(r, c)] - T * lt[IX(r, c - 1)] + (c < nx ? T * lt[IX(r, c)] : 0.0);
            lh_new[IX(r, c - 1)] += mu * dd[0];
            if (c < nx) lh_new[IX(r, c)] += mu * dd[1];
            lqx[IQX(r, c)] = mu * dd[2];
            if (c < nx) {
                grad_n[IX(r, c - 1)] += mu * dd[3] * scale * 0.5;
                grad_n[IX(r, c)] += mu * dd[3] * scale * 0.5;
                *grad_scale += mu * dd[3] * 0.5 * (n[IX(r, c - 1)] + n[IX(r, c)]);
            } else {
                grad_n[IX(r, c - 1)] += mu * dd[3] * scale;
                *grad_scale += mu * dd[3] * n[IX(r, c - 1)];
            }
        }
    for (int r = 0; r < ny; ++r) lqx[IQX(r, 0)] = 0.0;
    for (int r = 1; r <= ny; ++r)
        for (int c = 0; c < nx; ++c) {
            const double* dd = dy1 + IQY(r, c) * 4;
            double mu = lqy[IQY(r, c)] - T * lt[IX(r - 1, c)] + (r < ny ? T * lt[IX(r, c)] : 0.0);
            lh_new[IX(r - 1, c)] += mu * dd[0];
            if (r < ny) lh_new[IX(r, c)] += mu * dd[1];
            lqy[IQY(r, c)] = mu * dd[2];
            if (r < ny) {
                grad_n[IX(r - 1, c)] += mu * dd[3] * scale * 0.5;
                grad_n[IX(r, c)] += mu * dd[3] * scale * 0.5;
                *grad_scale += mu * dd[3] * 0.5 * (n[IX(r - 1, c)] + n[IX(r, c)]);
            } else {
                grad_n[IX(r - 1, c)] += mu * dd[3] * scale;
                *grad_scale += mu * dd[3] * n[IX(r - 1, c)];
            }
        }
    for (int c = 0; c < nx; ++c) lqy[IQY(0, c)] = 0.0;
    memcpy(lh, lh_new, sizeof(double) * (size_t)ny * nx);
    free(lh_new);
    free(qxn);
    free(qyn);
    free(dx1);
    free(dy1);
    free(lt);
}

/* Loss L = sum over sample times t_s = s * sample_dt (s = 1..ns) and gauges
 * g of (h(t_s)[cells[g]] - d[s-1][g])^2 for one member started from h0 (links
 * at rest) at t = 0, and its gradients: grad_n [ny*nx] (base Manning field),
 * grad_h0 [ny*nx], *grad_rain (rain multiplier), *grad_scale (Manning scale),
 * *grad_drain (land cover: the drainage field scaled by kappa, at kappa = 1).
 * Stores the whole trajectory (small grids only).  Returns the loss. */
double orc_loss_and_grad(const orc_params* p, const double* z, const double* n, double scale,
                         double rain_mult, const double* hyeto, int n_blocks, const double* h0,
                         double sample_dt, int ns, int G, const int32_t* cells, const double* d,
                         double* grad_n, double* grad_h0, double* grad_rain, double* grad_scale,
                         double* grad_drain, long* n_steps_out)
{
    const int ny = p->ny, nx = p->nx;
    const size_t nc = (size_t)ny * nx, nqx = (size_t)ny * (nx + 1), nqy = (size_t)(ny + 1) * nx;
    const size_t per = nc + nqx + nqy;
    long cap = 1024, nst = 0;
    double* traj = (double*)malloc(sizeof(double) * per * (size_t)(cap + 1));
    double* dts = (double*)malloc(sizeof(double) * (size_t)cap);
    double* rates = (double*)malloc(sizeof(double) * (size_t)cap);
    double* qins = (double*)malloc(sizeof(double) * (size_t)cap);   /* inflow flux per step */
    int* sample_after = (int*)malloc(sizeof(int) * (size_t)cap);   /* sample index or -1 */
    double* h = (double*)malloc(sizeof(double) * nc);
    double* qx = (double*)calloc(nqx, sizeof(double));
    double* qy = (double*)calloc(nqy, sizeof(double));
    double* qxs = (double*)malloc(sizeof(double) * nqx);
    double* qys = (double*)malloc(sizeof(double) * nqy);
    memcpy(h, h0, sizeof(double) * nc);
    orc_volumes vol = {0, 0, 0};
    double t = 0.0, loss = 0.0;
    for (int s = 1; s <= ns; ++s) {
        double t_end = s * sample_dt;
        while (t < t_end) {
            if (nst == cap) {
                cap *= 2;
                traj = (double*)realloc(traj, sizeof(double) * per * (size_t)(cap + 1));
                dts = (double*)realloc(dts, sizeof(double) * (size_t)cap);
                rates = (double*)realloc(rates, sizeof(double) * (size_t)cap);
                qins = (double*)realloc(qins, sizeof(double) * (size_t)cap);
                sample_after = (int*)realloc(sample_after, sizeof(int) * (size_t)cap);
            }
            double* st = traj + per * (size_t)nst;
            memcpy(st, h, sizeof(double) * nc);
            memcpy(st + nc, qx, sizeof(double) * nqx);
            memcpy(st + nc + nqx, qy, sizeof(double) * nqy);
            double t_next;
            double dt = orc_dt(p, orc_hmax(ny, nx, h), t, t_end, &t_next);
            double rate = orc_rain_rate(p, hyeto, n_blocks, t);
            orc_params ps = *p;
            if (p->inflow)
                ps.inflow_q = orc_rain_rate(p, p->inflow, p->inflow_blocks, t) /
                              (p->dx * (double)(p->inflow_r1 - p->inflow_r0));
            orc_step(&ps, z, n, scale, rate * rain_mult, dt, h, qx, qy, qxs, qys, &vol);
            dts[nst] = dt;
            rates[nst] = rate;
            qins[nst] = ps.inflow_q;
            sample_after[nst] = -1;
            t = t_next;
            ++nst;
        }
        sample_after[nst - 1] = s - 1;
        for (int g = 0; g < G; ++g) {
            double e = h[cells[g]] - d[(size_t)(s - 1) * G + g];
            loss += e * e;
        }
    }
    /* reverse sweep */
    double* lh = (double*)calloc(nc, sizeof(double));
    double* lqx = (double*)calloc(nqx, sizeof(double));
    double* lqy = (double*)calloc(nqy, sizeof(double));
    for (size_t i = 0; i < nc; ++i) grad_n[i] = 0.0;
    *grad_rain = 0.0;
    *grad_scale = 0.0;
    *grad_drain = 0.0;
    for (long k = nst - 1; k >= 0; --k) {
        if (sample_after[k] >= 0) {
            /* the state after step k is observed: h_{k+1} is the next stored
               state, or the final state for the last step */
            const double* hk1 = (k + 1 < nst) ? traj + per * (size_t)(k + 1) : h;
            int s = sample_after[k];
            for (int g = 0; g < G; ++g)
                lh[cells[g]] += 2.0 * (hk1[cells[g]] - d[(size_t)s * G + g]);
        }
        const double* st = traj + per * (size_t)k;
        orc_params ps = *p;
        ps.inflow_q = qins[k];
        orc_step_adjoint(&ps, z, n, scale, rates[k], rain_mult, dts[k], st, st + nc, st + nc + nqx,
                         lh, lqx, lqy, grad_n, grad_rain, grad_scale, grad_drain);
    }
    memcpy(grad_h0, lh, sizeof(double) * nc);
    if (n_steps_out) *n_steps_out = nst;
    free(lh); free(lqx); free(lqy); free(traj); free(dts); free(rates); free(qins); free(sample_after);
    free(h); free(qx); free(qy); free(qxs); free(qys);
    return loss;
}
