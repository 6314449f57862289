"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
the oracle's pins catch every one: a dropped term, a wrong sign, index or
exponent anywhere in Eq. 1-5, Eq. 4, Eq. 9-12 or the resampling must fail at
least one pin.  Each planted variant runs in its own process, so a variant
that crashes (an index run past the end) counts as caught too."""
import concurrent.futures as cf
import functools
import json
import os
import subprocess
import sys

import oracle
from tests import test_oracle_adjoint as A
from tests import test_oracle_helpers as H
from tests import test_oracle_inflow as IN
from tests import test_oracle_land_cover as LC
from tests import test_oracle_pf as P
from tests import test_oracle_scheme as S

PINS = [
    S.test_dt_matches_section_4_1_numbers,
    S.test_dt_floor_cap_fixed_and_event_clipping,
    S.test_two_cell_hand_steps,
    functools.partial(S.test_manning_normal_flow_is_fixed_point_of_eq2, dt=0.3),
    S.test_seiche_period_is_2L_over_sqrt_gH,
    S.test_lake_at_rest_over_bumpy_bed,
    S.test_uniform_rain_on_flat_closed_box,
    S.test_volume_balance_exact_to_1e12,
    S.test_transposition_symmetry,
    S.test_no_flow_over_a_dry_wall_eq3,
    S.test_shallow_sheet_below_h_eps_does_not_move,
    S.test_free_outflow_passes_outward_only,
    S.test_positivity_with_limiter_on_urban_dem,
    functools.partial(P.test_weights_match_scipy_gaussian_density, seed=0),
    P.test_relative_sigma_variant,
    P.test_equal_likelihood_keeps_prior_weights_and_neff_bounds,
    functools.partial(P.test_systematic_resampling_brute_force, M=5),
    P.test_one_hot_weights_select_one_particle,
    P.test_slot_assignment_keeps_survivors_in_place,
    A.test_gradients_match_central_differences_fully_wet,
    functools.partial(A.test_dot_product_identity_per_step, regime="wet"),
    functools.partial(A.test_dot_product_identity_per_step, regime="limited"),
    functools.partial(A.test_dot_product_identity_per_step, regime="drying"),
    functools.partial(A.test_dot_product_identity_per_step, regime="outflow"),
    functools.partial(A.test_dot_product_identity_per_step, regime="land_cover"),
    A.test_closed_form_uniform_rain_on_flat_box,
    LC.test_flat_box_rain_above_drainage_closed_form,
    LC.test_flat_box_drainage_above_rain_takes_all,
    LC.test_volume_balance_with_land_cover_exact_to_1e12,
    LC.test_wall_cells_stay_dry_and_pass_no_flow,
    LC.test_adjoint_with_land_cover_matches_central_differences,
    LC.test_adjoint_drainage_that_takes_everything_passes_nothing,
    LC.test_adjoint_flat_box_rain_above_drainage_closed_form,
    IN.test_closed_box_stores_the_inflow_exactly,
    IN.test_piecewise_series_lands_on_block_edges,
    IN.test_volume_balance_with_inflow_and_rain_to_1e12,
    H.test_steps_at_rest_take_eq4_of_section_4_1_depth,
    functools.partial(H.test_the_deepest_cell_decides_the_step, where=(5, 7)),
    H.test_gauge_sample_reads_the_member_and_cell_it_names,
    functools.partial(H.test_ensemble_loop_equals_each_member_alone, nthreads=4),
]

# (name, original text, planted mistake)
MUTATIONS = [
    ("friction exponent 4/3", "pow(hflow, -7.0 / 3.0)", "pow(hflow, -4.0 / 3.0)"),
    ("friction n instead of n^2", "p->g * nl * nl * dt * (fabs(q)", "p->g * nl * dt * (fabs(q)"),
    ("friction without dt", "p->g * nl * nl * dt * (fabs(q)", "p->g * nl * nl * (fabs(q)"),
    ("slope sign flipped", "(eta2 - eta1) / p->dx", "(eta1 - eta2) / p->dx"),
    ("gravity term without g", "q - p->g * hflow * dt * S", "q - hflow * dt * S"),
    ("Eq 3 as max depth", "fmax(eta1, eta2) - fmax(z1, z2)", "fmax(h1, h2)"),
    ("Eq 3 with min bed", "fmax(eta1, eta2) - fmax(z1, z2)", "fmax(eta1, eta2) - fmin(z1, z2)"),
    ("limiter on downstream depth", "(qn > 0.0 ? h1 : h2)", "(qn > 0.0 ? h2 : h1)"),
    ("Eq 5 drops the south link", "+ qy_new[IQY(r, c)] * dx - qy_new[IQY(r + 1, c)] * dx",
     "+ qy_new[IQY(r, c)] * dx"),
    ("Eq 5 x/y index swap", "qx_new[IQX(r, c)] * dx - qx_new[IQX(r, c + 1)] * dx",
     "qx_new[IQX(r, c)] * dx - qx_new[IQX(r, c)] * dx"),
    ("Eq 1 divides by dx only", "dt * dV / (dx * dx)", "dt * dV / dx"),
    ("rain without dt", "+ dt * rain * rcv;", "+ rain * rcv;"),
    ("runoff coefficient ignored", "+ dt * rain * rcv;", "+ dt * rain;"),
    ("drainage not limited by the water present", "if (sink > avail) sink = avail;", ""),
    ("drainage without dt", "double sink = dt * p->drain[IX(r, c)];",
     "double sink = p->drain[IX(r, c)];"),
    ("rain volume ignores the runoff coefficient", "area += p->rc[i];", "area += 1.0;"),
    ("inflow leaves instead of entering", "? p->inflow_q", "? -p->inflow_q"),
    ("inflow not spread over the segment", "(p->dx * (double)(p->inflow_r1 - p->inflow_r0))",
     "p->dx"),
    ("inflow volume not counted", "vol->inflow += dt * qx_new[IQX(r, 0)] * dx;", ""),
    ("x-link roughness not averaged", "scale * 0.5 * (n[IX(r, c - 1)] + n[IX(r, c)])",
     "scale * n[IX(r, c)]"),
    ("roughness scale dropped on y links", "double nl = scale * 0.5 * (n[IX(r - 1, c)]",
     "double nl = 0.5 * (n[IX(r - 1, c)]"),
    ("ghost cell dry", "orc_link_flux(p, h, z, h, z - p->edge_slope", "orc_link_flux(p, h, z, 0.0, z - p->edge_slope"),
    ("ghost cell above the edge", "z - p->edge_slope * p->dx", "z + p->edge_slope * p->dx"),
    ("Eq 4 without g", "sqrt(p->g * hm)", "sqrt(hm)"),
    ("Eq 4 ignores the cap", "if (dt > p->dt_cap) dt = p->dt_cap;", ""),
    ("no landing on the block edge", "if (t + dt >= stop) {", "if (0) {"),
    ("likelihood without the 1/2", "lw[i] = log(w_prior[i]) - 0.5 * chi2;",
     "lw[i] = log(w_prior[i]) - chi2;"),
    ("prior weight ignored", "lw[i] = log(w_prior[i]) - 0.5 * chi2;", "lw[i] = -0.5 * chi2;"),
    ("N_eff as 1/sum w", "s2 += w_post[i] * w_post[i];", "s2 += w_post[i];"),
    ("sigma not squared", "double e = (y[(size_t)i * G + g] - d[g]) / s;\n            chi2 += e * e;",
     "double e = (y[(size_t)i * G + g] - d[g]) / s;\n            chi2 += e * e * s;"),
    ("systematic offsets u + j/M", "double uj = (u + (double)j) / (double)M;",
     "double uj = u + (double)j / (double)M;"),
    ("resampling picks zero-weight ties", "c[i] <= uj) ++i;", "c[i] < uj) ++i;"),
    ("survivor slots not kept", "if (k[s] >= 1) {", "if (k[s] >= 2) {"),
    ("adjoint friction exponent", "-(7.0 / 3.0) * fric / hflow", "-(4.0 / 3.0) * fric / hflow"),
    ("adjoint slope sign", "*d_h1 = (first ? dq_dhf : 0.0) - dq_dS / p->dx;",
     "*d_h1 = (first ? dq_dhf : 0.0) + dq_dS / p->dx;"),
    ("adjoint clamp passes sensitivity", "lt[IX(r, c)] = pass ? lh[IX(r, c)] : 0.0;",
     "lt[IX(r, c)] = lh[IX(r, c)];"),
    ("adjoint drained cell passes sensitivity",
     "if (p->drain && hpre > 0.0 && hpre <= dt * p->drain[IX(r, c)]) pass = 0;", ""),
    ("adjoint drainage gradient without dt",
     "gk -= lt[IX(r, c)] * dt * p->drain[IX(r, c)];", "gk -= lt[IX(r, c)] * p->drain[IX(r, c)];"),
    ("adjoint drainage gradient with the wrong sign",
     "gk -= lt[IX(r, c)] * dt * p->drain[IX(r, c)];", "gk += lt[IX(r, c)] * dt * p->drain[IX(r, c)];"),
    ("adjoint rain gradient without the runoff coefficient",
     "gr += lt[IX(r, c)] * dt * rate * rcv;", "gr += lt[IX(r, c)] * dt * rate;"),
    ("adjoint limiter on the wrong cell", "*d_h1 = p->dx / (4.0 * dt);\n            return lim;",
     "*d_h2 = p->dx / (4.0 * dt);\n            return lim;"),
    ("adjoint continuity without dt/dx", "double mu = lqx[IQX(r, c)] - T * lt[IX(r, c - 1)]",
     "double mu = lqx[IQX(r, c)] - lt[IX(r, c - 1)]"),
    ("adjoint Manning gradient without scale",
     "grad_n[IX(r, c - 1)] += mu * dd[3] * scale * 0.5;\n                grad_n[IX(r, c)] += mu * dd[3] * scale * 0.5;",
     "grad_n[IX(r, c - 1)] += mu * dd[3] * 0.5;\n                grad_n[IX(r, c)] += mu * dd[3] * 0.5;"),
    ("adjoint ghost depth ignored", "dd[0] = a + b;   /* the ghost carries the edge depth */",
     "dd[0] = a;"),
    ("adjoint loss without the 2", "lh[cells[g]] += 2.0 * (hk1[cells[g]]",
     "lh[cells[g]] += (hk1[cells[g]]"),
    ("adjoint rain without dt", "gr += lt[IX(r, c)] * dt * rate * rcv;", "gr += lt[IX(r, c)] * rate * rcv;"),
    ("h_max over the first row only",
     "for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) m = h[i] > m ? h[i] : m;",
     "for (size_t i = 0; i < (size_t)nx; ++i) m = h[i] > m ? h[i] : m;"),
    ("h_max as the minimum", "m = h[i] > m ? h[i] : m;", "m = h[i] < m ? h[i] : m;"),
    ("h_max as the mean depth",
     "for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) m = h[i] > m ? h[i] : m;\n    return m;",
     "for (size_t i = 0; i < (size_t)ny * (size_t)nx; ++i) m += h[i];\n    return m / ((double)ny * nx);"),
    ("gauge member stride of the gauge count", "h[(size_t)m * ncell + cells[g]]",
     "h[(size_t)m * G + cells[g]]"),
    ("gauge outputs transposed", "y[(size_t)m * G + g] =", "y[(size_t)g * M + m] ="),
    ("ensemble qx offset by the cell count", "qx + m * nqx", "qx + m * nc"),
    ("ensemble members share one clock", "&t[m], t_end", "&t[0], t_end"),
    ("ensemble members share one scale", "scale[m], rain_mult[m]", "scale[0], rain_mult[m]"),
]




def run_pins(lib_path):
    """Run every pin against the oracle library at lib_path; return the names
    of the pins that failed."""
    oracle._lib = oracle.load(lib_path)
    failed = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError, FloatingPointError):
            failed.append(getattr(pin, "__name__", getattr(pin, "func", pin).__name__))
    return failed


def test_pins_catch_every_planted_mistake(tmp_path):
    src = oracle.source()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    jobs = []
    for k, (name, orig, bad) in enumerate(MUTATIONS):
        # the first occurrence is planted (the forward link flux comes before
        # its differentiated copy in the adjoint section)
        assert src.count(orig) >= 1, f"mutation anchor for {name!r} not found"
        path = oracle.compile_variant(src.replace(orig, bad, 1), str(tmp_path / f"libmut{k}.so"))
        jobs.append((name, path))

    def run(job):
        name, path = job
        code = ("import json, sys; from tests import test_oracle_mutations as T; "
                f"print(json.dumps(T.run_pins({path!r})))")
        r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True,
                           text=True, timeout=600)
        if r.returncode != 0:
            return name, ["<crashed>"]
        return name, json.loads(r.stdout.strip().splitlines()[-1])

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(ex.map(run, jobs))
    missed = [name for name, failed in results.items() if not failed]
    assert not missed, f"pins missed planted mistakes: {missed}"
    # the unmodified oracle passes every pin
    assert run_pins(oracle.build()) == []
