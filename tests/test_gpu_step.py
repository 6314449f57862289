"""GPU parity of the fused local-inertial step (Eq. 1-5, Eq. 4) against the
FP64 oracle, through the C ABI.  Tolerances: depth 1e-3 m and relative
volume 1e-5 at the end of a run (the bar the FP32 path is held to; the paper
saw at most 0.3 cm between single and double precision, Section 4.2); one
step from an identical state agrees to FP32 rounding."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_member_from_gpu, oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _run_pair(capi, z, n, hy, rm, sc, t_end, params=None, h0=None, M=None):
    """Run the GPU ensemble and the oracle members to t_end; return both."""
    ny, nx = z.shape
    p = params or capi.Params.default()
    M = M or len(rm)
    op = oracle_params(p, ny, nx)
    with capi.Grid(z, n, p) as g:
        g.ensemble_init(M, rm, sc, hy, h0=h0)
        g.advance_to(t_end)
        g.sync()
        gs = [g.get_state(m) for m in range(M)]
        mem = g.members()
        vol = g.volumes()
    outs = []
    for m in range(M):
        h0m = None if h0 is None else (h0[m] if np.ndim(h0) == 3 else h0)
        mo = oracle.Member.dry(ny, nx, h0m)
        oracle.advance(op, z, n, float(sc[m]), float(rm[m]), hy, mo, t_end=t_end)
        outs.append(mo)
    return gs, mem, vol, outs


def test_single_member_256_square_600s_matches_oracle(capi):
    """Single member, 256 x 256, 3 m cells, 50 mm/h for 600 s, Courant 0.7,
    closed walls with free outflow on the lowest (east) edge."""
    terr = synth.make_terrain(256, 256, seed=0)
    hy = synth.hyetograph_constant(50.0, 600.0)
    gs, mem, vol, outs = _run_pair(capi, terr.z, terr.n, hy, np.ones(1, np.float32),
                                   np.ones(1, np.float32), 600.0)
    h, qx, qy = gs[0]
    mo = outs[0]
    assert mem["t"][0] == 600.0 and mo.t == 600.0
    assert mem["steps"][0] == mo.steps
    err = compare(h, mo.h, 1e-3)
    V_gpu, V_or = vol["storage"][0], oracle.storage(mo.h, 3.0)
    assert abs(V_gpu - V_or) <= 1e-5 * V_or
    assert abs(vol["rain"][0] - mo.rain) <= 1e-6 * mo.rain
    assert abs(vol["outflow"][0] - mo.outflow) <= 1e-3 * mo.rain
    print(f"256^2 600 s: max|dh| {err:.2e} m, steps {mo.steps}")


def test_fixed_step_control_run(capi):
    """The paper's fixed 0.25 s step (Section 4.1) as a control: identical
    time grids on both sides."""
    terr = synth.make_terrain(128, 160, seed=3)
    hy = synth.hyetograph_constant(80.0, 300.0)
    p = capi.Params.default(dt_fixed=0.25)
    gs, mem, vol, outs = _run_pair(capi, terr.z, terr.n, hy, np.array([1.3], np.float32),
                                   np.array([0.8], np.float32), 300.0, params=p)
    assert mem["steps"][0] == 1200 == outs[0].steps
    compare(gs[0][0], outs[0].h, 1e-3)


@pytest.mark.parametrize("ny,nx", [(1, 1), (1, 2), (2, 1), (3, 3), (5, 7), (1, 131), (130, 1),
                                   (37, 129), (70, 300), (9, 257)])
def test_ragged_and_tiny_grids_one_step_from_random_state(capi, ny, nx):
    """One step from the same random wet state (FP32 values on both sides):
    every link and depth agrees to FP32 rounding, across warp spans (128
    columns), row strips, ragged edges and degenerate 1-cell grids."""
    rng = np.random.default_rng(ny * 1000 + nx)
    z = rng.uniform(0.0, 1.5, (ny, nx)).astype(np.float32)
    n = rng.uniform(0.02, 0.08, (ny, nx)).astype(np.float32)
    h = rng.uniform(0.0, 0.8, (ny, nx)).astype(np.float32)
    h[rng.random((ny, nx)) < 0.15] = 0.0
    qx = rng.normal(0.0, 0.05, (ny, nx)).astype(np.float32)
    qy = rng.normal(0.0, 0.05, (ny, nx)).astype(np.float32)
    qx[:, -1] = np.abs(qx[:, -1])   # the east edge is an outflow: outward only
    qy[-1, :] = 0.0                 # the south edge is a wall
    p = capi.Params.default(dt_fixed=0.2)
    hy = np.array([30.0 / 3.6e6], np.float32)
    with capi.Grid(z, n, p) as g:
        g.ensemble_init(1, np.array([1.1], np.float32), np.array([0.9], np.float32), hy)
        g.set_state(0, h, qx, qy)
        g.step(1)
        h1, qx1, qy1 = g.get_state(0)
    mo = oracle_member_from_gpu(h, qx, qy)
    op = oracle_params(p, ny, nx)
    oracle.step(op, z, n, 0.9, float(hy[0]) * 1.1, 0.2, mo)
    compare(qx1, mo.qx[:, 1:], 2e-5 + 0.0)
    compare(qy1, mo.qy[1:, :], 2e-5)
    compare(h1, mo.h, 5e-6)
    assert np.all(mo.qx[:, 0] == 0) and np.all(mo.qy[0, :] == 0)


def test_south_outflow_and_limiter_off_variants(capi):
    rng = np.random.default_rng(5)
    ny, nx = 41, 67
    z = (0.01 * np.arange(ny)[:, None] + rng.uniform(0, 0.2, (ny, nx))).astype(np.float32)
    n = np.full((ny, nx), 0.04, np.float32)
    h0 = rng.uniform(0.0, 0.4, (ny, nx)).astype(np.float32)
    for lim in (0, 1):
        p = capi.Params.default(east_outflow=0, south_outflow=1, limiter=lim, dt_cap=0.3)
        gs, mem, vol, outs = _run_pair(capi, z, n, np.zeros(1, np.float32),
                                       np.ones(1, np.float32), np.ones(1, np.float32), 60.0,
                                       params=p, h0=h0)
        compare(gs[0][0], outs[0].h, 1e-3)
        assert vol["outflow"][0] > 0
        assert abs(vol["outflow"][0] - outs[0].outflow) <= 1e-3 * max(outs[0].outflow, 1.0)


def test_lake_at_rest_exact_on_gpu(capi):
    rng = np.random.default_rng(7)
    ny, nx = 45, 150
    z = (rng.integers(0, 2600, (ny, nx)) * 2.0 ** -10).astype(np.float32)
    h = np.maximum(2.0 - z, 0.0).astype(np.float32)
    p = capi.Params.default(east_outflow=0)
    with capi.Grid(z, np.full((ny, nx), 0.05, np.float32), p) as g:
        g.ensemble_init(2, np.zeros(2, np.float32), np.ones(2, np.float32),
                        np.zeros(1, np.float32), h0=h)
        g.step(100)
        for m in range(2):
            h1, qx1, qy1 = g.get_state(m)
            assert np.array_equal(h1, h)
            assert not qx1.any() and not qy1.any()


def test_transposition_symmetry_is_bitwise_on_gpu(capi):
    terr = synth.make_terrain(72, 140, seed=9)
    hy = synth.hyetograph_constant(100.0, 300.0)
    pa = capi.Params.default(east_outflow=1, south_outflow=0)
    pb = capi.Params.default(east_outflow=0, south_outflow=1)
    with capi.Grid(terr.z, terr.n, pa) as a, capi.Grid(terr.z.T.copy(), terr.n.T.copy(), pb) as b:
        for g in (a, b):
            g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), hy)
            g.advance_to(240.0)
        ha, qxa, qya = a.get_state(0)
        hb, qxb, qyb = b.get_state(0)
    assert np.array_equal(ha, hb.T)
    assert np.array_equal(qxa, qyb.T) and np.array_equal(qya, qxb.T)


def test_two_runs_are_bitwise_identical(capi):
    terr = synth.make_terrain(96, 200, seed=4)
    hy = synth.hyetograph_constant(150.0, 600.0)
    rm, sc = synth.ensemble_prior(4, 6)
    res = []
    for _ in range(2):
        with capi.Grid(terr.z, terr.n) as g:
            g.ensemble_init(6, rm, sc, hy)
            g.advance_to(420.0)
            res.append([g.get_state(m) for m in range(6)] + [g.volumes()])
    for m in range(6):
        for k in range(3):
            assert np.array_equal(res[0][m][k], res[1][m][k])
    for key in ("storage", "rain", "outflow", "clamp"):
        assert np.array_equal(res[0][6][key], res[1][6][key])


def test_ensemble_members_each_match_oracle_and_conserve_volume(capi):
    """Per-member rain multiplier and Manning scale (Section 4.1's uncertain
    inputs) with per-member adaptive steps."""
    terr = synth.make_terrain(80, 150, seed=12)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    M = 9
    rm, sc = synth.ensemble_prior(12, M)
    rm = (rm * 3.0).astype(np.float32)   # heavier storm: deeper water, CFL-limited steps
    gs, mem, vol, outs = _run_pair(capi, terr.z, terr.n, hy, rm, sc, 1500.0)
    for m in range(M):
        compare(gs[m][0], outs[m].h, 1e-3)
        assert mem["t"][m] == 1500.0
        V = vol["storage"][m]
        Vo = oracle.storage(outs[m].h, 3.0)
        assert abs(V - Vo) <= 1e-5 * Vo
        bal = V - (vol["rain"][m] - vol["outflow"][m] + vol["clamp"][m])
        assert abs(bal) <= 1e-5 * vol["rain"][m]
        assert gs[m][0].min() >= 0.0
    assert len(set(mem["steps"].tolist())) > 1 or mem["steps"][0] == outs[0].steps


def test_nan_input_is_reported_at_sync(capi):
    """Host-side fault injection: a non-finite depth fed in through the ABI is
    flagged by the kernel and returned as FLOOD_ERR_NAN."""
    z = np.zeros((8, 8), np.float32)
    with capi.Grid(z, np.full((8, 8), 0.03, np.float32)) as g:
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), np.zeros(1, np.float32))
        h = np.full((8, 8), 0.1, np.float32)
        h[3, 4] = np.nan
        g.set_state(0, h)
        g.step(2)
        with pytest.raises(capi.FloodError) as e:
            g.sync()
        assert e.value.code == -5


def test_staged_tile_wait_that_runs_out_is_reported_and_recoverable(capi):
    """Failure detection without a fault: with a zero wait budget every TMA
    row wait of the step kernel is a single non-blocking test, which gives up
    on a row whose copy is still in flight; the
    kernel drains its own copies, records the timeout and returns, the next
    synchronising call reports FLOOD_ERR_TIMEOUT, and after
    flood_ensemble_init clears the error word the same grid runs the steps
    again to the same state as a fresh grid."""
    terr = synth.make_terrain(256, 256, seed=17)
    hy = synth.hyetograph_constant(80.0, 300.0)
    rm, sc = synth.ensemble_prior(17, 4)
    with capi.Grid(terr.z, terr.n) as ref:
        ref.ensemble_init(4, rm, sc, hy)
        ref.set_engine(1)
        ref.advance_to(30.0)
        want = [ref.get_state(m) for m in range(4)]
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(4, rm, sc, hy)
        g.set_engine(1)
        g.set_wait_budget(0)
        with pytest.raises(capi.FloodError) as e:
            g.advance_to(30.0)
        assert e.value.code == -4
        with pytest.raises(capi.FloodError) as e:
            g.sync()                       # sticky until the ensemble is initialised again
        assert e.value.code == -4
        g.set_wait_budget(-1)
        g.ensemble_init(4, rm, sc, hy)
        g.advance_to(30.0)
        for m in range(4):
            for k in range(3):
                assert np.array_equal(g.get_state(m)[k], want[m][k])


def test_bad_arguments_raise(capi):
    z = np.zeros((4, 4), np.float32)
    with capi.Grid(z, z + 0.03) as g:
        with pytest.raises(capi.FloodError):
            g.step(1)                                     # before ensemble_init
        g.ensemble_init(2, np.ones(2, np.float32), np.ones(2, np.float32), np.zeros(1, np.float32))
        with pytest.raises(capi.FloodError):
            g.gauge_sample(np.array([16], np.int32))      # cell out of range
        with pytest.raises(capi.FloodError):
            g.pf_assimilate(np.zeros(1), 0.05, 1.5, np.ones(2, np.float32))  # u outside [0,1)
        with pytest.raises(capi.FloodError):
            g.get_state(2)


def test_launch_shapes_give_bitwise_identical_results(capi):
    """The step kernel's launch shape (rows per strip, members per CTA) moves
    halo recomputation around but never changes a state value; the FP64
    volume bookkeeping sums FP32 per-warp partials, whose grouping follows the
    shape, so it agrees to ~1e-10 relative."""
    terr = synth.make_terrain(70, 300, seed=14)
    hy = synth.hyetograph_constant(120.0, 300.0)
    rm, sc = synth.ensemble_prior(14, 5)
    res = []
    for shape in [(0, 0), (1, 1), (3, 2), (16, 4), (64, 8), (128, 1)]:
        with capi.Grid(terr.z, terr.n) as g:
            g.ensemble_init(5, rm, sc, hy)
            g.set_launch(*shape)
            g.advance_to(90.0)
            g.set_launch(0, 0)
            g.advance_to(180.0)
            res.append(([g.get_state(m) for m in range(5)], g.volumes()))
    for states, vol in res[1:]:
        for m in range(5):
            for k in range(3):
                assert np.array_equal(states[m][k], res[0][0][m][k])
        for key in ("storage", "rain"):
            assert np.array_equal(vol[key], res[0][1][key])
        assert np.allclose(vol["outflow"], res[0][1]["outflow"], rtol=1e-8, atol=0)


def test_engines_give_bitwise_identical_results(capi):
    """Direct-load, TMA-staged and one-launch-per-member step kernels: same
    values, bit for bit, on a ragged grid (spans, strips and both grid edges
    exercised)."""
    terr = synth.make_terrain(75, 261, seed=15)
    hy = synth.hyetograph_constant(150.0, 300.0)
    rm, sc = synth.ensemble_prior(15, 6)
    res = []
    for engine, shape in [(0, (0, 0)), (1, (0, 0)), (1, (5, 1)), (1, (64, 4)), (0, (7, 4)),
                          (2, (0, 0)), (2, (16, 1))]:
        with capi.Grid(terr.z, terr.n) as g:
            g.ensemble_init(6, rm, sc, hy)
            g.set_engine(engine)
            g.set_launch(*shape)
            g.advance_to(150.0)
            g.sync()
            res.append(([g.get_state(m) for m in range(6)], g.members()["steps"]))
    for states, steps in res[1:]:
        assert np.array_equal(steps, res[0][1])
        for m in range(6):
            for k in range(3):
                assert np.array_equal(states[m][k], res[0][0][m][k])


def test_autotune_leaves_the_ensemble_untouched(capi):
    """The autotuner times real steps on the live ensemble, then restores it:
    the run continues exactly as if it had never been tuned."""
    terr = synth.make_terrain(90, 300, seed=16)
    hy = synth.hyetograph_constant(150.0, 600.0)
    rm, sc = synth.ensemble_prior(16, 8)
    res = []
    for tune in (False, True):
        with capi.Grid(terr.z, terr.n) as g:
            g.ensemble_init(8, rm, sc, hy)
            g.advance_to(120.0)
            before = g.members()
            if tune:
                rows, mpc, eng, ms = g.autotune(steps_per_trial=3)
                assert rows in (32, 64, 128) and mpc in (1, 4) and eng in (0, 1) and ms > 0
                after = g.members()
                assert np.array_equal(before["t"], after["t"])
                assert np.array_equal(before["steps"], after["steps"])
            g.advance_to(300.0)
            res.append(([g.get_state(m) for m in range(8)], g.volumes(), g.members()))
    for m in range(8):
        for k in range(3):
            assert np.array_equal(res[0][0][m][k], res[1][0][m][k])
    assert np.array_equal(res[0][1]["rain"], res[1][1]["rain"])
    assert np.allclose(res[0][1]["outflow"], res[1][1]["outflow"], rtol=1e-8, atol=0)
    assert np.array_equal(res[0][2]["steps"], res[1][2]["steps"])


@pytest.mark.parametrize("ny,nx", [(37, 129), (70, 300), (5, 7)])
def test_wet_dry_threshold_one_step_on_dyadic_state(capi, ny, nx):
    """h_eps = 1e-3 m (links whose flow depth is at most 1 mm carry no flow):
    one step from the same state on both sides.  Beds are multiples of
    2^-10 m and depths multiples of 2^-14 m, most of them within a few mm of
    the threshold, so Eq. 3's flow depth is exact in FP32 and FP64 and both
    sides switch the same links off; every link and depth then agrees to
    FP32 rounding, and the threshold is seen to act (links the default
    h_eps = 0 lets flow carry none here)."""
    rng = np.random.default_rng(ny * 7 + nx)
    z = (rng.integers(0, 1536, (ny, nx)) / 1024.0).astype(np.float32)
    n = rng.uniform(0.02, 0.08, (ny, nx)).astype(np.float32)
    h = (rng.integers(0, 80, (ny, nx)) / 16384.0).astype(np.float32)
    deep = rng.random((ny, nx)) < 0.3
    h[deep] = (rng.integers(0, 8192, deep.sum()) / 16384.0).astype(np.float32)
    qx = rng.normal(0.0, 0.01, (ny, nx)).astype(np.float32)
    qy = rng.normal(0.0, 0.01, (ny, nx)).astype(np.float32)
    qx[:, -1] = np.abs(qx[:, -1])
    qy[-1, :] = 0.0
    p = capi.Params.default(dt_fixed=0.2, h_eps=1e-3)
    hy = np.array([30.0 / 3.6e6], np.float32)
    with capi.Grid(z, n, p) as g:
        g.ensemble_init(1, np.array([1.1], np.float32), np.array([0.9], np.float32), hy)
        g.set_state(0, h, qx, qy)
        g.step(1)
        h1, qx1, qy1 = g.get_state(0)
    op = oracle_params(p, ny, nx)
    assert op.h_eps == 1e-3
    mo = oracle_member_from_gpu(h, qx, qy)
    oracle.step(op, z, n, 0.9, float(hy[0]) * 1.1, 0.2, mo)
    compare(qx1, mo.qx[:, 1:], 2e-5)
    compare(qy1, mo.qy[1:, :], 2e-5)
    compare(h1, mo.h, 5e-6)
    # the links the threshold switched off: zero on both sides, flowing without it
    op0 = oracle_params(capi.Params.default(dt_fixed=0.2), ny, nx)
    m0 = oracle_member_from_gpu(h, qx, qy)
    oracle.step(op0, z, n, 0.9, float(hy[0]) * 1.1, 0.2, m0)
    off = (mo.qx[:, 1:] == 0.0) & (m0.qx[:, 1:] != 0.0)
    assert off.sum() >= 1 and np.all(qx1[off] == 0.0)
