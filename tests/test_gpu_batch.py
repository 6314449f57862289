"""GPU uneven batches (flood_batch_*, extension beyond the paper): scenarios
of different grid sizes, storms and durations advanced together, each
matching the FP64 oracle and, bit for bit, the same scenario run alone."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_params, require_gpu

pytestmark = pytest.mark.gpu

SHAPES = [(37, 53), (64, 64), (130, 97), (20, 260), (90, 129)]


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _scenarios():
    rng = np.random.default_rng(77)
    terrs = [synth.make_terrain(ny, nx, seed=100 + k) for k, (ny, nx) in enumerate(SHAPES)]
    durations = [300.0, 450.0, 600.0, 375.0, 510.0]
    rates = rng.uniform(20.0, 100.0, len(SHAPES))
    hys = [synth.hyetograph_constant(r, t) for r, t in zip(rates, durations)]
    rm = rng.uniform(0.8, 1.5, len(SHAPES)).astype(np.float32)
    sc = rng.uniform(0.7, 1.3, len(SHAPES)).astype(np.float32)
    return terrs, hys, rm, sc, np.array(durations)


def _run_batch(capi, shape=None, engine=None):
    terrs, hys, rm, sc, dur = _scenarios()
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        b.init(hys, rm, sc, dur)
        if shape:
            b.set_launch(*shape)
        if engine is not None:
            b.set_engine(engine)
        for w in (300.0, 600.0):
            b.step(w)
        states = [b.get_state(i) for i in range(len(SHAPES))]
        mem = b.members()
    return terrs, hys, rm, sc, dur, states, mem


def test_batch_matches_oracle_and_single_runs(capi):
    terrs, hys, rm, sc, dur, states, mem = _run_batch(capi)
    assert np.array_equal(mem["t"], dur)
    assert len(set(mem["steps"].tolist())) > 1
    p = capi.Params.default()
    for i, t in enumerate(terrs):
        ny, nx = t.z.shape
        mo = oracle.Member.dry(ny, nx)
        oracle.advance(oracle_params(p, ny, nx), t.z, t.n, float(sc[i]), float(rm[i]), hys[i], mo,
                       t_end=float(dur[i]))
        compare(states[i][0], mo.h, 1e-3)
        assert mem["steps"][i] == mo.steps
        V = mem["storage"][i]
        assert abs(V - oracle.storage(mo.h, p.dx)) <= 1e-5 * oracle.storage(mo.h, p.dx)
        assert abs(V - (mem["rain"][i] - mem["outflow"][i] + mem["clamp"][i])) <= 1e-5 * mem["rain"][i]
        with capi.Grid(t.z, t.n, p) as g:
            g.ensemble_init(1, rm[i:i + 1], sc[i:i + 1], hys[i])
            g.advance_to(float(dur[i]))
            alone = g.get_state(0)
        for k in range(3):
            assert np.array_equal(states[i][k], alone[k])


@pytest.mark.parametrize("shape", [(1, 4), (16, 8), (200, 4)])
def test_batch_launch_shapes_bitwise(capi, shape):
    ref = _run_batch(capi)[5]
    got = _run_batch(capi, shape)[5]
    for a, b in zip(ref, got):
        for k in range(3):
            assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("shape", [None, (7, 8)])
def test_batch_engines_bitwise(capi, shape):
    """Direct-load and TMA-staged batched kernels, graph-replayed or in one
    persistent launch: the same states, bit for bit, for every scenario, and
    the same clocks and volume bookkeeping."""
    runs = [_run_batch(capi, shape, engine=e) for e in (0, 1, 2)]
    for r in runs[1:]:
        for x, y in zip(runs[0][5], r[5]):
            for k in range(3):
                assert np.array_equal(x[k], y[k])
        for key in ("t", "steps", "rain", "outflow", "clamp", "storage"):
            assert np.array_equal(runs[1][6][key], r[6][key]), key


def test_persistent_batch_runs_windows_in_one_launch_each(capi):
    """The persistent engine advances a window in one launch (plus nothing
    else on the device), and scenarios that already ended stay put."""
    terrs, hys, rm, sc, dur = _scenarios()
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        b.init(hys, rm, sc, dur)
        b.set_engine(2)
        n0 = b.launch_count
        b.step(300.0)
        assert b.launch_count - n0 == 1
        t1 = b.members()["t"]
        assert np.array_equal(t1, np.minimum(dur, 300.0))
        b.step(300.0)                     # nothing left to do: no launch
        assert b.launch_count - n0 == 1
        b.step(1000.0)
        assert np.array_equal(b.members()["t"], dur)


def test_batch_autotune_leaves_the_batch_unchanged(capi):
    """The batched-step autotuner times its candidates on the live batch and
    puts it back: continuing after the tuning reaches the same states, clocks
    and rain, bit for bit, as a run that was never tuned."""
    terrs, hys, rm, sc, dur = _scenarios()
    res = []
    for tune in (False, True):
        with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
            b.init(hys, rm, sc, dur)
            b.step(300.0)
            if tune:
                rows, warps, engine, ms = b.autotune(20.0)
                assert rows in (16, 32, 64) and warps in (4, 8) and engine in (1, 2) and ms > 0
            b.step(600.0)
            res.append(([b.get_state(i) for i in range(len(SHAPES))], b.members()))
    for x, y in zip(res[0][0], res[1][0]):
        for k in range(3):
            assert np.array_equal(x[k], y[k])
    for key in ("t", "steps", "rain"):
        assert np.array_equal(res[0][1][key], res[1][1][key]), key
    for key in ("outflow", "clamp", "storage"):
        assert np.allclose(res[0][1][key], res[1][1][key], rtol=1e-9, atol=1e-12), key


def test_persistent_barrier_wait_that_runs_out_is_reported_and_recoverable(capi):
    """Failure detection of the persistent form without a fault: with a zero
    barrier budget every CTA that is not the last to arrive gives up at
    once; the step call returns FLOOD_ERR_TIMEOUT, and after flood_batch_init
    the same batch runs to a fresh batch's states bit for bit."""
    terrs, hys, rm, sc, dur = _scenarios()
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as ref:
        ref.init(hys, rm, sc, dur)
        ref.set_engine(2)
        ref.step(300.0)
        want = [ref.get_state(i) for i in range(len(SHAPES))]
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        b.init(hys, rm, sc, dur)
        b.set_engine(2)
        b.set_wait_budget(0)
        with pytest.raises(capi.FloodError) as e:
            b.step(300.0)
        assert e.value.code == -4
        b.set_wait_budget(-1)
        b.init(hys, rm, sc, dur)
        b.step(300.0)
        for i in range(len(SHAPES)):
            for k in range(3):
                assert np.array_equal(b.get_state(i)[k], want[i][k])


def test_batch_rejects_bad_arguments(capi):
    z = np.zeros((4, 4), np.float32)
    with pytest.raises(capi.FloodError):
        capi.Batch([z, np.zeros((0, 3), np.float32)], [z, np.zeros((0, 3), np.float32)])
    with capi.Batch([z], [z + 0.03]) as b:
        with pytest.raises(capi.FloodError):
            b.step(10.0)        # before init
        with pytest.raises(capi.FloodError):
            b.set_launch(0, 4)


def test_full_size_uneven_batch_to_the_end_follows_the_oracle(capi):
    """The uneven batch at its real size: 64 square scenarios of 512^2 to
    2048^2 cells (108 M in all), rain 20-100 mm/h, 900-3600 s, advanced in
    300 s windows by the persistent launch with the tuner's 32-row strips
    until every scenario has ended.  The smallest scenario (520^2, 1733 s)
    and a mid-size one (1085^2, 1094 s) against the FP64 oracle over their
    whole duration: depth 1e-3 m, storage 1e-5 relative, the same number
    of steps; every scenario's own balance to 1e-5 of its rain."""
    import concurrent.futures as cf
    scen = synth.uneven_batch(64)
    terrs = [synth.make_terrain(s.ny, s.nx, seed=s.seed) for s in scen]
    hys = [synth.hyetograph_constant(s.rain_mm_h, s.duration_s) for s in scen]
    dur = np.array([s.duration_s for s in scen])
    ones = np.ones(len(scen), np.float32)
    picks = (27, 20)
    assert (scen[27].ny, scen[20].ny) == (520, 1085)
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        b.set_engine(2)
        b.set_launch(32, 4)
        b.init(hys, ones, ones, dur)
        for w in range(1, 13):
            b.step(300.0 * w)
        mem = b.members()
        states = {i: b.get_state(i)[0] for i in picks}
    assert np.array_equal(mem["t"], dur)
    bal = mem["storage"] - (mem["rain"] - mem["outflow"] + mem["clamp"])
    assert np.all(np.abs(bal) <= 1e-5 * mem["rain"])
    p = capi.Params.default()

    def run(i):
        ny, nx = terrs[i].z.shape
        mo = oracle.Member.dry(ny, nx)
        oracle.advance(oracle_params(p, ny, nx), terrs[i].z, terrs[i].n, 1.0, 1.0, hys[i], mo,
                       t_end=float(dur[i]))
        return mo

    with cf.ThreadPoolExecutor(max_workers=len(picks)) as ex:   # the oracle releases the GIL
        ref = dict(zip(picks, ex.map(run, picks)))
    for i in picks:
        err = compare(states[i], ref[i].h, 1e-3)
        V = oracle.storage(ref[i].h, p.dx)
        assert abs(mem["storage"][i] - V) <= 1e-5 * V
        assert mem["steps"][i] == ref[i].steps
        print(f"batch scenario {i} ({scen[i].ny}^2, {dur[i]:.0f} s): max |dh| {err:.2e} m, "
              f"storage rel err {abs(mem['storage'][i] - V) / V:.2e}, {ref[i].steps} steps")


@pytest.mark.parametrize("engine", [0, 1, 2])
def test_batch_with_several_members_per_scenario(capi, engine):
    """Scenarios with 1-4 members each (an ensemble per scenario, every
    member with its own rain multiplier, Manning scale, state, clock and
    step length): every member equals, bit for bit, the same member of a
    single-grid ensemble of its scenario; the batch's per-member volumes
    close their balance; one member follows the FP64 oracle."""
    terrs, hys, rm1, sc1, dur = _scenarios()
    counts = np.array([1, 4, 2, 3, 4], np.int32)
    rng = np.random.default_rng(78)
    rm = rng.uniform(0.7, 1.6, counts.sum()).astype(np.float32)
    sc = rng.uniform(0.7, 1.3, counts.sum()).astype(np.float32)
    first = np.concatenate([[0], np.cumsum(counts)])
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        b.set_engine(engine)
        b.init(hys, rm, sc, dur, members=counts)
        for w in (300.0, 600.0):
            b.step(w)
        got = {(i, m): b.get_state(i, member=m) for i in range(len(SHAPES)) for m in range(counts[i])}
        mem = b.members()
    assert mem["t"].shape == (counts.sum(),)
    assert np.array_equal(mem["t"], np.repeat(dur, counts))
    bal = mem["storage"] - (mem["rain"] - mem["outflow"] + mem["clamp"])
    assert np.all(np.abs(bal) <= 1e-5 * mem["rain"])
    p = capi.Params.default()
    for i, t in enumerate(terrs):
        sl = slice(first[i], first[i + 1])
        with capi.Grid(t.z, t.n, p) as g:
            g.ensemble_init(int(counts[i]), rm[sl], sc[sl], hys[i])
            g.advance_to(float(dur[i]))
            steps = g.members()["steps"]
            for m in range(counts[i]):
                alone = g.get_state(m)
                for k in range(3):
                    assert np.array_equal(got[(i, m)][k], alone[k]), (i, m, k)
        assert np.array_equal(mem["steps"][sl], steps)
    # one member of the four-member scenario against the oracle
    i, m = 1, 2
    ny, nx = terrs[i].z.shape
    mo = oracle.Member.dry(ny, nx)
    oracle.advance(oracle_params(p, ny, nx), terrs[i].z, terrs[i].n, float(sc[first[i] + m]),
                   float(rm[first[i] + m]), hys[i], mo, t_end=float(dur[i]))
    compare(got[(i, m)][0], mo.h, 1e-3)


@pytest.mark.parametrize("engine", [0, 1, 2])
def test_batch_with_land_cover(capi, engine):
    """Land cover in the batch (Section 4.1): three scenarios of uneven sizes
    with per-class roughness, runoff and drainage, cells outside the domain
    (two western quarter discs, and an irregular domain whose outside tiles
    are not scheduled), two or three members each with their own class
    roughness and drainage rate.  Every member equals, bit for bit, the same
    member of a single-grid land-cover ensemble of its scenario (same step
    counts; drained volumes to the rounding of per-strip partials); the balance closes with
    the drained volume; one member follows the FP64 oracle."""
    shapes = [(70, 150), (45, 260), (150, 300)]
    terrs = [synth.make_terrain(ny, nx, seed=120 + k) for k, (ny, nx) in enumerate(shapes)]
    clss = [synth.land_cover(terrs[0], seed=121, pond_side=(6, 14)),
            synth.land_cover(terrs[1], seed=122, pond_side=(5, 12)),
            synth.land_cover(terrs[2], seed=123, pond_side=(6, 14),
                             domain=synth.irregular_domain(150, 300, 0.55, seed=123))]
    counts = np.array([2, 3, 2], np.int32)
    first = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(124)
    rm = rng.uniform(0.8, 1.5, counts.sum()).astype(np.float32)
    sc = rng.uniform(0.8, 1.2, counts.sum()).astype(np.float32)
    n_cls = [(np.array([c[0] for c in synth.LAND_CLASSES], np.float32)
              * rng.uniform(0.7, 1.4, (counts[i], 4))).astype(np.float32) for i in range(3)]
    drain = [rng.uniform(5.0, 20.0, counts[i]).astype(np.float32) / 3.6e6 for i in range(3)]
    dur = np.array([600.0, 450.0, 540.0])
    hys = [synth.hyetograph_constant(r, t) for r, t in zip((120.0, 80.0, 150.0), dur)]
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        for i in range(3):
            b.set_land_cover(i, clss[i], synth.LAND_CLASSES)
        b.set_engine(engine)
        b.init(hys, rm, sc, dur, members=counts)
        for i in range(3):
            b.set_land_params(i, n_cls[i], drain[i])
        for w in (300.0, 600.0):
            b.step(w)
        got = {(i, m): b.get_state(i, member=m) for i in range(3) for m in range(counts[i])}
        mem = b.members()
        drained = b.drained()
    assert np.array_equal(mem["t"], np.repeat(dur, counts))
    assert np.all(drained > 0)
    bal = mem["storage"] - (mem["rain"] - mem["outflow"] + mem["clamp"] - drained)
    assert np.all(np.abs(bal) <= 1e-5 * mem["rain"])
    p = capi.Params.default()
    for i, t in enumerate(terrs):
        sl = slice(first[i], first[i + 1])
        with capi.Grid(t.z, t.n, p) as g:
            g.set_land_cover(clss[i], synth.LAND_CLASSES)
            g.ensemble_init(int(counts[i]), rm[sl], sc[sl], hys[i])
            g.set_land_params(n_cls[i], drain[i])
            g.advance_to(float(dur[i]))
            members = g.members()
            vols = g.volumes()
            for m in range(counts[i]):
                alone = g.get_state(m)
                for k in range(3):
                    assert np.array_equal(got[(i, m)][k], alone[k]), (i, m, k)
            grid_drained = g.drained()
        assert np.array_equal(mem["steps"][sl], members["steps"])
        # per-warp FP32 partials over the rows of each strip: the launch shapes differ
        assert np.allclose(drained[sl], grid_drained, rtol=1e-8, atol=0)
        assert np.allclose(mem["rain"][sl], vols["rain"], rtol=1e-12, atol=0)
    # the irregular domain: cells outside it stay dry and at rest
    out = ~synth.irregular_domain(150, 300, 0.55, seed=123)
    for m in range(counts[2]):
        assert np.all(got[(2, m)][0][out] == 0) and np.all(got[(2, m)][1][out] == 0)
    # one member against the oracle
    i, m = 0, 1
    tab = synth.LAND_CLASSES
    outside = np.array([c[3] for c in tab], bool)
    runoff = np.where(outside, 0.0, np.array([c[1] for c in tab], np.float32)).astype(np.float64)
    drains = np.where(outside, 0, np.array([c[2] for c in tab])).astype(np.float64)
    cls = clss[i]
    z = np.where(outside[cls], np.float32(1.0e6), terrs[i].z).astype(np.float32)
    n = n_cls[i][m][cls].astype(np.float64)
    ny, nx = z.shape
    op = oracle_params(p, ny, nx)
    op.rc = np.ascontiguousarray(runoff[cls])
    op.drain = np.ascontiguousarray(float(np.float32(drain[i][m])) * drains[cls])
    mo = oracle.Member.dry(ny, nx)
    oracle.advance(op, z, n, float(sc[first[i] + m]), float(rm[first[i] + m]), hys[i], mo,
                   t_end=float(dur[i]))
    compare(got[(i, m)][0], mo.h, 1e-3)
    assert mo.drained > 0 and abs(drained[first[i] + m] - mo.drained) <= 1e-3 * mo.drained


def test_batch_land_cover_refusals(capi):
    terrs = [synth.make_terrain(20, 30, seed=130 + k) for k in range(2)]
    cls = synth.land_cover(terrs[0], seed=130, pond_side=(3, 5))
    hy = synth.hyetograph_constant(50.0, 300.0)
    with capi.Batch([t.z for t in terrs], [t.n for t in terrs]) as b:
        with pytest.raises(capi.FloodError):
            b.set_land_cover(2, cls, synth.LAND_CLASSES)          # no such scenario
        with pytest.raises(capi.FloodError):
            b.set_land_cover(0, cls + 4, synth.LAND_CLASSES)      # class out of range
        b.set_land_cover(0, cls, synth.LAND_CLASSES)
        with pytest.raises(capi.FloodError):
            b.set_land_cover(0, cls, synth.LAND_CLASSES)          # set twice
        with pytest.raises(capi.FloodError):                      # one scenario of two
            b.init([hy, hy], np.ones(2, np.float32), np.ones(2, np.float32), [300.0, 300.0])
        b.set_land_cover(1, synth.land_cover(terrs[1], seed=131, pond_side=(3, 5)),
                         synth.LAND_CLASSES)
        b.init([hy, hy], np.ones(2, np.float32), np.ones(2, np.float32), [300.0, 300.0])
        with pytest.raises(capi.FloodError):
            b.set_land_cover(0, cls, synth.LAND_CLASSES)          # after init
        with pytest.raises(capi.FloodError):
            b.set_land_params(0, -np.ones((1, 4), np.float32))    # roughness must be positive
