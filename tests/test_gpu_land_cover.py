"""GPU land cover (Section 4.1, Table 1): per-class roughness and runoff
coefficient, drainage on hardened ground, cells outside the domain, with
the per-member class roughness and drainage rate as the ensemble's
uncertain inputs; against the FP64 oracle, bit for bit across engines and
launch shapes, through a resampling, and at the full 2000 x 2000 x 96 size
on sampled patches."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_member_from_gpu, oracle_params, require_gpu

pytestmark = pytest.mark.gpu

WALL_Z = np.float32(1.0e6)


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _oracle_fields(terr, cls, n_m, drain_m):
    """The fields the oracle needs for one member, from the same FP32 inputs
    the device uses."""
    tab = synth.LAND_CLASSES
    outside = np.array([c[3] for c in tab], bool)
    runoff = np.where(outside, 0.0, np.array([c[1] for c in tab], np.float32)).astype(np.float64)
    drains = np.where(outside, 0, np.array([c[2] for c in tab])).astype(np.float64)
    z = np.where(outside[cls], WALL_Z, terr.z).astype(np.float32)
    n = np.asarray(n_m, np.float32)[cls].astype(np.float64)
    rc = runoff[cls]
    dr = float(np.float32(drain_m)) * drains[cls]
    return z, n, np.ascontiguousarray(rc), np.ascontiguousarray(dr), outside[cls]


def _run(capi, terr, cls, hy, rm, sc, n_m, d_m, t_end, engine=None, shape=None, params=None):
    M = len(rm)
    with capi.Grid(terr.z, terr.n, params) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy)
        g.set_land_params(n_m, d_m)
        if engine is not None:
            g.set_engine(engine)
        if shape is not None:
            g.set_launch(*shape)
        g.advance_to(t_end)
        g.sync()
        states = [g.get_state(m) for m in range(M)]
        return states, g.members(), g.volumes(), g.drained()


def test_land_cover_follows_the_oracle(capi):
    ny, nx, M = 64, 100, 3
    terr = synth.make_terrain(ny, nx, seed=61)
    cls = synth.land_cover(terr, seed=61, pond_side=(6, 14))
    assert set(np.unique(cls)) == {0, 1, 2, 3}
    hy = synth.hyetograph_constant(100.0, 600.0)
    rm, sc = synth.ensemble_prior(61, M)
    n_m, d_m = synth.land_prior(61, M)
    p = capi.Params.default()
    states, mem, vol, drained = _run(capi, terr, cls, hy, rm, sc, n_m, d_m, 600.0, params=p)
    for m in range(M):
        z, n, rc, dr, out = _oracle_fields(terr, cls, n_m[m], d_m[m])
        op = oracle_params(p, ny, nx)
        op.rc, op.drain = rc, dr
        mo = oracle.Member.dry(ny, nx)
        oracle.advance(op, z, n, float(sc[m]), float(rm[m]), hy, mo, t_end=600.0)
        h = states[m][0]
        compare(h, mo.h, 1e-3)
        assert np.all(h[out] == 0.0) and np.all(mo.h[out] == 0.0)
        assert mo.drained > 0
        assert abs(drained[m] - mo.drained) <= 1e-3 * mo.drained
        assert abs(vol["rain"][m] - mo.rain) <= 1e-6 * mo.rain
        V = vol["storage"][m]
        assert abs(V - oracle.storage(mo.h, p.dx)) <= 1e-5 * oracle.storage(mo.h, p.dx)
        bal = V - (vol["rain"][m] - vol["outflow"][m] + vol["clamp"][m] - drained[m])
        assert abs(bal) <= 1e-5 * vol["rain"][m]


@pytest.mark.parametrize("case", [(0, (16, 4)), (0, (7, 1)), (1, (0, 0)), (1, (5, 1)), (1, (64, 4))])
def test_land_cover_engines_and_shapes_bitwise(capi, case):
    ny, nx, M = 45, 150, 5
    terr = synth.make_terrain(ny, nx, seed=62)
    cls = synth.land_cover(terr, seed=62, pond_side=(5, 12))
    hy = synth.hyetograph_constant(120.0, 300.0)
    rm, sc = synth.ensemble_prior(62, M)
    n_m, d_m = synth.land_prior(62, M)
    ref = _run(capi, terr, cls, hy, rm, sc, n_m, d_m, 240.0, engine=1)
    got = _run(capi, terr, cls, hy, rm, sc, n_m, d_m, 240.0, engine=case[0], shape=case[1])
    for m in range(M):
        for k in range(3):
            assert np.array_equal(got[0][m][k], ref[0][m][k])
    assert np.array_equal(got[1]["steps"], ref[1]["steps"])
    assert np.allclose(got[3], ref[3], rtol=1e-8, atol=0)


@pytest.mark.parametrize("engine", [0, 1])
def test_tracked_maximum_with_land_cover(capi, engine):
    """Land cover with the running maximum tracked (the TMA form then stages
    the maxima and the class bytes in the same row stage): the maxima are
    bit for bit the maximum of the stepped states, and the states equal the
    untracked run's."""
    ny, nx, M = 45, 150, 5
    terr = synth.make_terrain(ny, nx, seed=63)
    cls = synth.land_cover(terr, seed=63, pond_side=(5, 12))
    hy = synth.hyetograph_constant(120.0, 300.0)
    rm, sc = synth.ensemble_prior(63, M)
    n_m, d_m = synth.land_prior(63, M)
    p = capi.Params.default(dt_fixed=0.5)
    plain = _run(capi, terr, cls, hy, rm, sc, n_m, d_m, 40.0, engine=engine, params=p)[0]
    with capi.Grid(terr.z, terr.n, p) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy)
        g.set_land_params(n_m, d_m)
        g.set_engine(engine)
        g.advance_to(20.0)
        g.track_max_depth(True)
        host = np.array([g.get_state(m)[0] for m in range(M)])
        for _ in range(40):
            g.step(1)
            host = np.maximum(host, np.array([g.get_state(m)[0] for m in range(M)]))
        got = np.array([g.max_depth(m) for m in range(M)])
        states = [g.get_state(m) for m in range(M)]
    assert np.array_equal(got, host)
    for m in range(M):
        for k in range(3):
            assert np.array_equal(states[m][k], plain[m][k])


def test_resampling_carries_land_parameters(capi):
    ny, nx, M = 32, 48, 6
    terr = synth.make_terrain(ny, nx, seed=63)
    cls = synth.land_cover(terr, seed=63, pond_side=(4, 8))
    hy = synth.hyetograph_constant(80.0, 300.0)
    rm, sc = synth.ensemble_prior(63, M)
    n_m, d_m = synth.land_prior(63, M)
    with capi.Grid(terr.z, terr.n) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy)
        g.set_land_params(n_m, d_m)
        g.advance_to(120.0)
        y = g.gauge_sample(np.array([5 * nx + 30, 20 * nx + 40], np.int32))
        u, beta = synth.pf_draws(63, 1, M)
        # a sharp observation of member 2: the resampling duplicates it
        pf = g.pf_assimilate(y[2].astype(np.float64), 0.001, u, beta, force=True)
        n2, d2 = g.land_params()
    src = oracle.assign_slots(pf["idx"])
    assert len(set(src.tolist())) < M
    assert np.array_equal(n2, n_m[src]) and np.array_equal(d2, d_m[src])


def test_land_cover_refusals(capi):
    terr = synth.make_terrain(24, 30, seed=64)
    cls = synth.land_cover(terr, seed=64, pond_side=(3, 5))
    hy = synth.hyetograph_constant(50.0, 300.0)
    with capi.Grid(terr.z, terr.n) as g:
        bad = cls.copy(); bad[0, 0] = 7
        with pytest.raises(capi.FloodError):
            g.set_land_cover(bad, synth.LAND_CLASSES)
        g.set_land_cover(cls, synth.LAND_CLASSES)
        with pytest.raises(capi.FloodError):
            g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(2, np.ones(2, np.float32), np.ones(2, np.float32), hy)
        with pytest.raises(capi.FloodError):
            g.set_land_params(drain_rate=np.array([-1.0, 0.0], np.float32))


def test_full_size_land_cover_window(capi):
    """2000 x 2000 cells, 96 members with their own class roughness and
    drainage, one 300 s window of the triangular storm in the benchmark's
    launch configuration: the volume balance of every member, the outside
    cells dry, and one further step against the oracle on sampled patches of
    three members."""
    ny = nx = 2000
    M = 96
    terr = synth.make_terrain(ny, nx, seed=1)
    cls = synth.land_cover(terr, seed=1)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(1, M)
    n_m, d_m = synth.land_prior(1, M)
    p = capi.Params.default()
    sample = [0, 47, 95]
    with capi.Grid(terr.z, terr.n, p) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy)
        g.set_land_params(n_m, d_m)
        g.advance_to(300.0)
        g.sync()
        vol = g.volumes()
        drained = g.drained()
        bal = vol["storage"] - (vol["rain"] - vol["outflow"] + vol["clamp"] - drained)
        assert np.all(np.abs(bal) <= 1e-5 * vol["rain"])
        assert np.all(drained > 0)
        mem0 = g.members()
        before = {m: g.get_state(m) for m in sample}
        g.step(1)
        mem1 = g.members()
        after = {m: g.get_state(m) for m in sample}
    rng = np.random.default_rng(2)
    for m in sample:
        dt = mem1["t"][m] - mem0["t"][m]
        h, qx, qy = before[m]
        z, n, rc, dr, out = _oracle_fields(terr, cls, n_m[m], d_m[m])
        assert np.all(h[out] == 0.0) and h.min() >= 0.0
        for (rc0, cc0) in [tuple(rng.integers(40, 1960, 2)) for _ in range(2)]:
            r0, r1, c0, c1 = rc0 - 33, rc0 + 33, cc0 - 33, cc0 + 33
            sub = oracle_params(p, r1 - r0, c1 - c0)
            sub.east_outflow = 0
            sub.rc = np.ascontiguousarray(rc[r0:r1, c0:c1])
            sub.drain = np.ascontiguousarray(dr[r0:r1, c0:c1])
            mo = oracle_member_from_gpu(h[r0:r1, c0:c1], qx[r0:r1, c0:c1], qy[r0:r1, c0:c1])
            rate = float(hy[1]) if mem0["t"][m] >= 300.0 else float(hy[0])
            oracle.step(sub, z[r0:r1, c0:c1], n[r0:r1, c0:c1], float(sc[m]), rate * float(rm[m]),
                        dt, mo)
            compare(after[m][0][r0:r1, c0:c1][1:-1, 1:-1], mo.h[1:-1, 1:-1], 2e-5)


def test_irregular_domain_skips_outside_tiles_and_follows_the_oracle(capi):
    """An irregular domain shaped like the paper's study area (Section 4.1:
    the active cells fill 58 % of their bounding box), here 40 % of a
    130 x 530 box so that many 128-column x 8-row tiles lie wholly outside
    it.  The ordinary TMA step launches only the tiles that hold a cell of
    the domain; the direct-load engine launches them all: both give the same
    states, clocks and volumes bit for bit, and the oracle (which evolves
    every cell) agrees.  Water given for cells outside the domain, at the
    start or by flood_set_state, is dropped: those cells stay dry and at
    rest."""
    ny, nx, M = 130, 530, 3
    terr = synth.make_terrain(ny, nx, seed=64)
    dom = synth.irregular_domain(ny, nx, 0.40, seed=64)
    cls = synth.land_cover(terr, seed=64, pond_side=(5, 12), domain=dom)
    out_cell = cls == 3
    R = 8
    tiles_in = sum(dom[a:a + R, b:b + 128].any() for a in range(0, ny, R) for b in range(0, nx, 128))
    tiles_all = ((ny + R - 1) // R) * ((nx + 127) // 128)
    assert tiles_in <= 0.7 * tiles_all
    hy = synth.hyetograph_constant(100.0, 600.0)
    rm, sc = synth.ensemble_prior(64, M)
    n_m, d_m = synth.land_prior(64, M)
    h0 = np.full((ny, nx), 0.02, np.float32)          # water everywhere, outside cells too
    p = capi.Params.default()
    res = []
    for engine in (1, 0):
        with capi.Grid(terr.z, terr.n, p) as g:
            g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(M, rm, sc, hy, h0=h0)
            g.set_land_params(n_m, d_m)
            g.set_engine(engine)
            g.set_launch(R, 1)
            start = g.get_state(1)
            assert np.all(start[0][out_cell] == 0.0) and np.all(start[0][~out_cell] == 0.02)
            g.advance_to(300.0)
            hh, qx, qy = g.get_state(1)
            g.set_state(1, hh + 0.01, qx + 0.001, qy)  # outside cells: dropped again
            g.advance_to(600.0)
            g.sync()
            res.append(([g.get_state(m) for m in range(M)], g.members(), g.volumes(), g.drained()))
    (st1, mem1, vol1, dr1), (st0, mem0, vol0, dr0) = res
    for m in range(M):
        for k in range(3):
            assert np.array_equal(st1[m][k], st0[m][k]), (m, k)
        assert np.all(st1[m][0][out_cell] == 0.0) and np.all(st1[m][1][out_cell] == 0.0)
    assert np.array_equal(mem1["steps"], mem0["steps"]) and np.array_equal(mem1["t"], mem0["t"])
    for key in ("storage", "rain", "outflow", "clamp"):
        assert np.allclose(vol1[key], vol0[key], rtol=1e-9, atol=1e-9), key
    # the oracle from the same start (member 0 and 2: no set_state in between)
    for m in (0, 2):
        z, n, rc, dr, out = _oracle_fields(terr, cls, n_m[m], d_m[m])
        op = oracle_params(p, ny, nx)
        op.rc, op.drain = rc, dr
        mo = oracle.Member.dry(ny, nx, np.where(out, 0.0, 0.02))
        oracle.advance(op, z, n, float(sc[m]), float(rm[m]), hy, mo, t_end=600.0)
        compare(st1[m][0], mo.h, 1e-3)
        assert np.all(mo.h[out] == 0.0)
        V = oracle.storage(mo.h, p.dx)
        assert abs(vol1["storage"][m] - V) <= 1e-5 * V


def test_water_body_warmup_follows_the_oracle(capi):
    """§4.1's start: the water bodies filled to a 3.0 m water level, then a
    warm-up with no rain (shortened here to 600 s), through the initial depth
    field of the ensemble: against the oracle from the same field, the volume
    balance closing with the drainage and the outflow."""
    ny, nx, M = 64, 100, 2
    terr = synth.make_terrain(ny, nx, seed=64)
    cls = synth.land_cover(terr, seed=64, pond_side=(6, 14))
    water = cls == 1
    assert water.any()
    h0 = np.where(water, np.maximum(np.float32(3.0) - terr.z, 0.0), 0.0).astype(np.float32)
    assert h0.max() > 0
    hy = synth.hyetograph_constant(0.0, 600.0)
    rm, sc = synth.ensemble_prior(64, M)
    n_m, d_m = synth.land_prior(64, M)
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy, h0=h0)
        g.set_land_params(n_m, d_m)
        V0 = g.volumes()["storage"]
        g.advance_to(600.0)
        states = [g.get_state(m) for m in range(M)]
        vol = g.volumes()
        drained = g.drained()
    for m in range(M):
        z, n, rc, dr, out = _oracle_fields(terr, cls, n_m[m], d_m[m])
        op = oracle_params(p, ny, nx)
        op.rc, op.drain = rc, dr
        mo = oracle.Member.dry(ny, nx)
        mo.h[:] = np.where(out, 0.0, h0)
        oracle.advance(op, z, n, float(sc[m]), float(rm[m]), hy, mo, t_end=600.0)
        compare(states[m][0], mo.h, 1e-3)
        assert vol["rain"][m] == 0.0
        bal = vol["storage"][m] - (V0[m] - vol["outflow"][m] + vol["clamp"][m] - drained[m])
        assert abs(bal) <= 1e-5 * V0[m]
