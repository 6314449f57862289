"""GPU parity of the particle filter (Eq. 9-12, systematic resampling, DA
steps (I)-(V) of Section 3.3, perturbation of Section 4.4) against the FP64
oracle: weights within 1e-6 relative, resampled indices bit-exact, state
replacement exact.  Plus an ensemble run with assimilation windows and a
sampled check at the full 2000 x 2000 x 96 size."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_member_from_gpu, oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


@pytest.mark.parametrize("M", [1, 2, 7, 96, 1000])
def test_resampling_indices_bit_exact_given_oracle_weights(capi, M):
    rng = np.random.default_rng(M)
    for trial in range(25):
        w = rng.dirichlet(np.ones(M) * (0.1 if trial % 2 else 2.0))
        u = float(rng.random()) if trial else 0.0
        assert np.array_equal(capi.resample_systematic(w, u), oracle.resample_systematic(w, u))
    w = np.zeros(M); w[M // 2] = 1.0
    assert np.all(capi.resample_systematic(w, 0.0) == M // 2)


def _ensemble(capi, M, ny=48, nx=70, seed=1):
    terr = synth.make_terrain(ny, nx, seed=seed)
    rm, sc = synth.ensemble_prior(seed, M)
    g = capi.Grid(terr.z, terr.n)
    g.ensemble_init(M, rm, sc, synth.hyetograph_constant(200.0, 600.0))
    g.advance_to(120.0)
    return g, terr, rm, sc


@pytest.mark.parametrize("M,force", [(12, False), (12, True), (96, False), (96, True)])
def test_weights_neff_and_replacement_match_oracle(capi, M, force):
    g, terr, rm, sc = _ensemble(capi, M)
    with g:
        cells = synth.gauge_cells(terr, 6, seed=3)
        y = g.gauge_sample(cells)
        before = [g.get_state(m) for m in range(M)]
        mem0 = g.members()
        # observations near one member so the weights degenerate
        d = y[M // 3].astype(np.float64) + 0.01
        u, beta = synth.pf_draws(7, 1, M)
        pf = g.pf_assimilate(d, 0.05, u, beta, force=force)
        after = [g.get_state(m) for m in range(M)]
        mem1 = g.members()
    ens = oracle.Ensemble(oracle.Params(ny=terr.z.shape[0], nx=terr.z.shape[1]), M)
    ens.h = np.stack([b[0] for b in before]).astype(np.float64)
    w_o, neff_o, idx_o, rm_o, sc_o = oracle.pf_assimilate(
        ens, y.astype(np.float64), d, np.full(6, 0.05), mem0["rain_mult"], mem0["scale"], u,
        beta, force=force)
    # oracle on the same inputs: weights within 1e-6 relative, N_eff likewise
    big = w_o > 1e-300
    assert np.allclose(pf["weights"][big], w_o[big], rtol=1e-6, atol=0)
    assert np.all(pf["weights"][~big] <= 1e-290)
    assert abs(pf["neff"] - neff_o) <= 1e-6 * neff_o
    assert pf["resampled"] == (idx_o is not None)
    if idx_o is None:
        assert np.array_equal(pf["idx"], np.arange(M))
        assert np.allclose(mem1["weights"], w_o, rtol=1e-6, atol=1e-300)
        for m in range(M):
            assert np.array_equal(after[m][0], before[m][0])
        return
    assert np.array_equal(pf["idx"], idx_o)
    src = oracle.assign_slots(idx_o)
    for s in range(M):
        for k in range(3):
            assert np.array_equal(after[s][k], before[src[s]][k])
    assert np.array_equal(mem1["rain_mult"], (mem0["rain_mult"][src] * beta).astype(np.float32))
    assert np.array_equal(mem1["scale"], mem0["scale"][src])
    assert np.allclose(mem1["weights"], 1.0 / M)
    assert np.allclose(mem1["rain_mult"], rm_o, rtol=1e-6)


def test_relative_sigma_and_supplied_outputs(capi):
    M = 10
    g, terr, rm, sc = _ensemble(capi, M, seed=2)
    with g:
        cells = synth.gauge_cells(terr, 4, seed=1)
        y = g.gauge_sample(cells)
        d = (y.mean(axis=0) + 0.02).astype(np.float64)
        y_in = (y + 0.003 * np.arange(M)[:, None]).astype(np.float32)
        pf = g.pf_assimilate(d, None, 0.25, np.ones(M, np.float32), y=y_in, sigma_rel=0.05,
                             n_thr_frac=0.0)
    w_o, neff_o = oracle.pf_weights(y_in.astype(np.float64), d, np.ones(4), np.full(M, 1 / M),
                                    sigma_rel=0.05)
    assert not pf["resampled"]
    assert np.allclose(pf["weights"], w_o, rtol=1e-6, atol=1e-300)


def test_assimilation_windows_follow_the_oracle(capi):
    """A reduced version of the ensemble + particle filter experiment: M
    members, a triangular storm, depth gauges at ponding spots, a hidden
    truth member (oracle) observed with N(0, 0.05^2) noise, assimilation
    every 300 s.  At each window the GPU ensemble is compared with the
    oracle ensemble; the oracle applies the resampling computed from the
    GPU's own gauge outputs (so both ensembles keep the same particles) and
    the indices must be bit-identical to the oracle's from those outputs."""
    ny, nx, M, G = 64, 96, 16, 6
    terr = synth.make_terrain(ny, nx, seed=21)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(21, M)
    rm = (rm * 4.0).astype(np.float32)
    cells = synth.gauge_cells(terr, G, seed=21)
    p = capi.Params.default()
    op = oracle_params(p, ny, nx)
    # hidden truth from the oracle with its own prior draw
    trm, tsc = synth.ensemble_prior(999, 1)
    truth = oracle.Member.dry(ny, nx)
    ens = oracle.Ensemble(op, M)
    rm_o = rm.astype(np.float64); sc_o = sc.astype(np.float64)
    resampled_any = False
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(M, rm, sc, hy)
        for wdw in range(1, 5):
            t = 300.0 * wdw
            g.advance_to(t)
            ens.advance(terr.z, terr.n, sc_o, rm_o, hy, t_end=t)
            oracle.advance(op, terr.z, terr.n, float(tsc[0]), float(trm[0] * 4.0), hy, truth,
                           t_end=t)
            d = synth.observe(truth.h.ravel()[cells], seed=21, window=wdw)
            y = g.gauge_sample(cells)
            for m in range(M):
                compare(g.get_state(m)[0], ens.h[m], 1e-3)
            y_o = oracle.gauge_sample(ens.h, cells)
            assert np.max(np.abs(y - y_o)) <= 1e-3
            u, beta = synth.pf_draws(21, wdw, M)
            mem = g.members()
            pf = g.pf_assimilate(d, 0.05, u, beta)
            # oracle PF on the GPU's outputs: same particles on both sides
            w_o, neff_o, idx_o, rm_new, sc_new = oracle.pf_assimilate(
                ens, y.astype(np.float64), d, np.full(G, 0.05), mem["rain_mult"], mem["scale"],
                u, beta)
            big = w_o > 1e-300
            assert np.allclose(pf["weights"][big], w_o[big], rtol=1e-6)
            assert pf["resampled"] == (idx_o is not None)
            if idx_o is not None:
                resampled_any = True
                assert np.array_equal(pf["idx"], idx_o)
                rm_o, sc_o = rm_new, sc_new
            # the oracle's weights from its own outputs stay close (FP32 vs FP64 state)
            w_own, _ = oracle.pf_weights(y_o, d, np.full(G, 0.05), np.full(M, 1.0 / M))
            assert np.isfinite(w_own).all()
        mem = g.members()
        assert np.allclose(mem["rain_mult"], rm_o, rtol=1e-6)
    assert resampled_any


def test_full_size_ensemble_sampled_parity(capi):
    """The full ensemble (2000 x 2000 cells, 96 members): advance one 300 s
    window in the benchmark's launch configuration, then check sampled
    outputs: one further GPU step against one oracle step from the same
    FP32 state on patches of three members, exact landing on 300 s, volume
    balance and non-negative depths for every member."""
    ny = nx = 2000
    M = 96
    terr = synth.make_terrain(ny, nx, seed=1)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(1, M)
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.advance_to(300.0)
        g.sync()
        mem0 = g.members()
        assert np.all(mem0["t"] == 300.0)
        vol = g.volumes()
        bal = vol["storage"] - (vol["rain"] - vol["outflow"] + vol["clamp"])
        assert np.all(np.abs(bal) <= 1e-5 * vol["rain"])
        sample = [0, 47, 95]
        before = {m: g.get_state(m) for m in sample}
        g.step(1)
        mem1 = g.members()
        after = {m: g.get_state(m) for m in sample}
    rng = np.random.default_rng(0)
    for m in sample:
        dt = mem1["t"][m] - mem0["t"][m]
        assert dt > 0
        h, qx, qy = before[m]
        assert h.min() >= 0.0
        # busiest patch (most water) plus a random one, each with a 1-cell halo
        wet = np.argwhere(h > 0.05)
        centres = [tuple(wet[len(wet) // 2]) if len(wet) else (1000, 1000),
                   tuple(rng.integers(40, 1960, 2))]
        for (rc, cc) in centres:
            r0, r1 = max(0, rc - 33), min(ny, rc + 33)
            c0, c1 = max(0, cc - 33), min(nx, cc + 33)
            sub = oracle_params(p, r1 - r0, c1 - c0)
            sub.east_outflow = 1 if c1 == nx else 0
            sub.south_outflow = 0
            mo = oracle_member_from_gpu(h[r0:r1, c0:c1], qx[r0:r1, c0:c1], qy[r0:r1, c0:c1])
            rate = float(hy[1]) if mem0["t"][m] >= 300.0 else float(hy[0])
            oracle.step(sub, terr.z[r0:r1, c0:c1], terr.n[r0:r1, c0:c1], float(sc[m]),
                        rate * float(rm[m]), dt, mo)
            # interior cells only: their four links lie inside the patch
            ha = after[m][0][r0:r1, c0:c1]
            compare(ha[1:-1, 1:-1], mo.h[1:-1, 1:-1], 2e-5)
            compare(after[m][1][r0:r1, c0:c1][1:-1, :-1], mo.qx[1:-1, 1:-1], 5e-5)


def test_resume_at_a_window_boundary_is_bit_exact(capi):
    """Checkpoint / resume through the ABI: the states, clocks, rain
    multipliers, Manning scales and weights read out at a window boundary
    (after the particle filter) and fed to a new grid (ensemble_init with
    per-member depths and the saved time, set_state, set_members) continue
    to exactly the states of the run that was never interrupted."""
    ny, nx, M = 64, 96, 6
    terr = synth.make_terrain(ny, nx, seed=21)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(21, M)
    cells = synth.gauge_cells(terr, 3, seed=21)
    u, beta = synth.pf_draws(21, 1, M)

    def first_window(g):
        g.ensemble_init(M, rm, sc, hy)
        g.advance_to(300.0)
        y = g.gauge_sample(cells)
        d = y.astype(np.float64).mean(axis=0) * 1.1
        g.pf_assimilate(d, 0.05, u, beta, y=y, force=True)

    with capi.Grid(terr.z, terr.n) as a:
        first_window(a)
        a.advance_to(600.0)
        want = [a.get_state(m) for m in range(M)]
        want_mem = a.members()
    with capi.Grid(terr.z, terr.n) as b:
        first_window(b)
        saved = [b.get_state(m) for m in range(M)]
        mem = b.members()
    assert np.all(mem["t"] == 300.0)
    with capi.Grid(terr.z, terr.n) as c:
        c.ensemble_init(M, mem["rain_mult"], mem["scale"], hy,
                        h0=np.stack([s[0] for s in saved]), t0=300.0)
        for m in range(M):
            c.set_state(m, *saved[m])
        c.set_members(weights=mem["weights"])
        c.advance_to(600.0)
        got = [c.get_state(m) for m in range(M)]
        got_mem = c.members()
    for m in range(M):
        for k in range(3):
            assert np.array_equal(got[m][k], want[m][k]), (m, k)
    assert np.array_equal(got_mem["t"], want_mem["t"])
    assert np.array_equal(got_mem["weights"], want_mem["weights"])
