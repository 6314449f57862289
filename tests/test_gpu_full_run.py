"""End-of-run parity of the ensemble at full size and full length: 2000 x 2000
cells of 3 m, 96 members, the 1 h triangular storm in twelve 300 s
assimilation windows with the particle filter after each (Section 3.3,
Fig. 5; the benchmark's workload), against the FP64 oracle.

The oracle cannot carry 96 full-size members through the hour in a test, so
it follows particles: every particle alive at the end descends, window by
window, from one of the initial particles (a resampling copies a state
exactly), so its whole ancestry can be evolved by the oracle from the dry
start at t = 0 with no restart; six final particles are followed, one host
thread each.  The resampling decisions the oracle takes
are its own -- Eq. 9-12 and systematic resampling on the GPU's gauge outputs
(the only outputs that exist for all 96 members), which must give the GPU's
indices bit for bit -- and the rain multipliers it carries are its own FP64
products of the caller's perturbations (Section 4.4).  The GPU run is
deterministic, so a second pass reads the ancestors' states at every window
end for the per-window comparison.  Bars: max |dh| <= 1e-3 m and storage
within 1e-5 relative of the oracle's at every window end (paper Section 4.2
compares FP32 with FP64 the same way); weights 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import oracle_params, require_gpu

pytestmark = pytest.mark.gpu

NY = NX = 2000
M, G, SEED, WINDOWS, WINDOW = 96, 6, 1, 12, 300.0
FOLLOW = (0, 19, 38, 57, 76, 95)   # final slots whose ancestry the oracle evolves


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _observations(capi, terr, hy, cells):
    """The benchmark's hidden truth: a member of its own prior draw, observed
    at the gauges with N(0, 0.05^2) noise at every window end."""
    trm, tsc = synth.ensemble_prior(SEED + 1000, 1)
    obs = []
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(1, trm, tsc, hy)
        for w in range(1, WINDOWS + 1):
            g.advance_to(WINDOW * w)
            obs.append(synth.observe(g.gauge_sample(cells)[0], seed=SEED, window=w))
    return obs


def _gpu_run(capi, terr, hy, rm, sc, cells, obs, read=None):
    """The twelve windows as the benchmark runs them.  read(w) -> slots whose
    depths to keep at the end of window w (before its filter update)."""
    rec = dict(y=[], pf=[], mem=[], kept={})
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        for w in range(1, WINDOWS + 1):
            g.advance_to(WINDOW * w)
            y = g.gauge_sample(cells)
            for s in (read(w) if read else ()):
                rec["kept"][(w, s)] = g.get_state(s)[0]
            u, beta = synth.pf_draws(SEED, w, M)
            rec["y"].append(y)
            rec["pf"].append(g.pf_assimilate(obs[w - 1], 0.05, u, beta))
            rec["mem"].append(g.members())
        g.sync()
        rec["final"] = {f: g.get_state(f)[0] for f in FOLLOW}
        rec["vol"] = g.volumes()
    return rec


def test_headline_ensemble_follows_the_oracle_for_the_whole_hour(capi):
    terr = synth.make_terrain(NY, NX, seed=SEED)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(SEED, M)
    cells = synth.gauge_cells(terr, G, seed=SEED)
    obs = _observations(capi, terr, hy, cells)
    run1 = _gpu_run(capi, terr, hy, rm, sc, cells, obs)

    # the oracle's filter on the GPU's outputs: weights, indices, slot maps,
    # and the rain multiplier / Manning scale every slot carries into the
    # next window
    w_prior = np.full(M, 1.0 / M)
    rm_o, sc_o = rm.astype(np.float64), sc.astype(np.float64)
    carried = [(rm_o.copy(), sc_o.copy())]      # parameters during window w + 1
    src_of = []                                  # slot map of each window's update
    n_resampled = 0
    for w in range(1, WINDOWS + 1):
        u, beta = synth.pf_draws(SEED, w, M)
        y = run1["y"][w - 1].astype(np.float64)
        wts, neff = oracle.pf_weights(y, obs[w - 1], np.full(G, 0.05), w_prior)
        pf = run1["pf"][w - 1]
        big = wts > 1e-300
        assert np.allclose(pf["weights"][big], wts[big], rtol=1e-6), w
        if neff < 0.8 * M:
            idx = oracle.resample_systematic(wts, u)
            assert pf["resampled"] and np.array_equal(pf["idx"], idx), w
            src = oracle.assign_slots(idx)
            rm_o = rm_o[src] * beta.astype(np.float64)
            sc_o = sc_o[src]
            w_prior = np.full(M, 1.0 / M)
            n_resampled += 1
        else:
            assert not pf["resampled"], w
            src = np.arange(M, dtype=np.int32)
            w_prior = wts
        src_of.append(src)
        carried.append((rm_o.copy(), sc_o.copy()))
        mem = run1["mem"][w - 1]
        assert np.allclose(mem["rain_mult"], rm_o, rtol=1e-6), w
        assert np.array_equal(mem["scale"], sc_o.astype(np.float32)), w
    assert n_resampled >= 1

    # ancestry of each followed final slot: the slot it occupied during window w
    during = {f: [0] * (WINDOWS + 1) for f in FOLLOW}
    for f in FOLLOW:
        a = f
        for w in range(WINDOWS, 0, -1):
            a = int(src_of[w - 1][a])
            during[f][w] = a

    run2 = _gpu_run(capi, terr, hy, rm, sc, cells, obs,
                    read=lambda w: sorted({during[f][w] for f in FOLLOW}))
    for f in FOLLOW:    # the GPU run repeats itself bit for bit
        assert np.array_equal(run2["final"][f], run1["final"][f])

    # the oracle evolves the followed ancestries from the dry start, one host
    # thread each
    op = oracle_params(capi.Params.default(), NY, NX)
    ens = oracle.Ensemble(op, len(FOLLOW))
    z = terr.z.astype(np.float64); n = terr.n.astype(np.float64)
    hy64 = hy.astype(np.float64)
    worst_h, worst_v = 0.0, 0.0
    for w in range(1, WINDOWS + 1):
        slots = [during[f][w] for f in FOLLOW]
        rmw, scw = carried[w - 1]
        ens.advance(z, n, scw[slots], rmw[slots], hy64, t_end=WINDOW * w, nthreads=len(FOLLOW))
        assert np.all(ens.t == WINDOW * w)
        for k, s in enumerate(slots):
            h_gpu = run2["kept"][(w, s)]
            err = float(np.max(np.abs(h_gpu.astype(np.float64) - ens.h[k])))
            v_o = oracle.storage(ens.h[k], op.dx)
            v_g = oracle.storage(h_gpu.astype(np.float64), op.dx)
            verr = abs(v_g - v_o) / v_o
            worst_h, worst_v = max(worst_h, err), max(worst_v, verr)
            assert err <= 1e-3, (w, s, err)
            assert verr <= 1e-5, (w, s, verr)
            y_gpu = run1["y"][w - 1][s]
            assert np.max(np.abs(y_gpu - ens.h[k].ravel()[cells])) <= 1e-3
    # end of run: the followed final slots hold the oracle's states
    for k, f in enumerate(FOLLOW):
        assert np.max(np.abs(run1["final"][f] - ens.h[k])) <= 1e-3
        v_o = oracle.storage(ens.h[k], op.dx)
        assert abs(run1["vol"]["storage"][f] - v_o) <= 1e-5 * v_o
    starts = sorted({during[f][1] for f in FOLLOW})
    print(f"full-run parity: {n_resampled} resamplings, max |dh| {worst_h:.3e} m, "
          f"max storage rel err {worst_v:.3e}, initial particles {starts}, ancestries "
          f"{ {f: during[f][1:] for f in FOLLOW} }")
