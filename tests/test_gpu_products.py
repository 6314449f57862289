"""GPU ensemble products (Section 4.4, Figs. 15-16): the running maximum
depth kept by the step kernels (bit for bit the maximum of the stepped
states, through a resampling that moves histories with their particles),
against the FP64 oracle's trajectory, and the exceedance / percentile maps
against the oracle's products of the same maxima and weights (bit for
bit), up to the full 2000 x 2000 x 96 ensemble on sampled rows."""
import numpy as np
import pytest

import oracle
from oracle import products as prod
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


@pytest.mark.parametrize("engine", [0, 1])
def test_tracked_maximum_is_the_maximum_of_the_steps(capi, engine):
    ny, nx, M = 45, 150, 5
    terr = synth.make_terrain(ny, nx, seed=51)
    hy = synth.hyetograph_constant(120.0, 600.0)
    rm, sc = synth.ensemble_prior(51, M)
    p = capi.Params.default(dt_fixed=0.5)   # members stay in step with one another
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.set_engine(engine)
        g.advance_to(60.0)
        g.track_max_depth(True)
        host = np.array([g.get_state(m)[0] for m in range(M)])
        for i in range(40):
            g.step(1)
            host = np.maximum(host, np.array([g.get_state(m)[0] for m in range(M)]))
            if i == 20:   # a forced resampling moves each particle's history with it
                y = g.gauge_sample(np.array([5 * nx + 7, 30 * nx + 100], np.int32))
                u, beta = synth.pf_draws(51, 1, M)
                pf = g.pf_assimilate(y[0].astype(np.float64), 0.05, u, beta, force=True)
                src = oracle.assign_slots(pf["idx"])
                host = host[src]
        got = np.array([g.max_depth(m) for m in range(M)])
    assert np.array_equal(got, host)


def test_maximum_follows_the_oracle_trajectory(capi):
    ny, nx = 64, 96
    terr = synth.make_terrain(ny, nx, seed=52)
    hy = synth.hyetograph_constant(80.0, 600.0)
    p = capi.Params.default(dt_fixed=0.5)
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), hy)
        g.track_max_depth(True)
        g.advance_to(300.0)
        got = g.max_depth(0)
    op = oracle_params(p, ny, nx)
    mo = oracle.Member.dry(ny, nx)
    hmax = mo.h.copy()
    for _ in range(600):
        oracle.advance(op, terr.z, terr.n, 1.0, 1.0, hy, mo, max_steps=1)
        hmax = prod.running_max(hmax, mo.h)
    assert mo.t == 300.0
    compare(got, hmax, 1e-3)


def test_products_equal_the_oracle_products_of_the_same_maxima(capi):
    ny, nx, M = 40, 70, 12
    terr = synth.make_terrain(ny, nx, seed=53)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(53, M)
    rm = (rm * 3.0).astype(np.float32)
    cells = synth.gauge_cells(terr, 4, seed=53)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.track_max_depth(True)
        g.advance_to(600.0)
        y = g.gauge_sample(cells)
        u, beta = synth.pf_draws(53, 1, M)
        # no resampling: the weights stay unequal
        g.pf_assimilate(y[3].astype(np.float64), 0.05, u, beta, n_thr_frac=1e-9)
        w = g.members()["weights"]
        levels = (0.1, 0.25, 0.5, 0.9, 1.0)
        exceed, pct = g.ensemble_products(0.05, levels)
        hm = np.array([g.max_depth(m) for m in range(M)])
    assert np.ptp(w) > 0
    assert np.array_equal(exceed, prod.exceedance(hm, w, 0.05))
    assert np.array_equal(pct, prod.percentiles(hm, w, levels))
    assert 0 < exceed.max() <= 1.0


def test_products_refuse_bad_calls(capi):
    terr = synth.make_terrain(16, 20, seed=54)
    hy = synth.hyetograph_constant(50.0, 300.0)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(2, np.ones(2, np.float32), np.ones(2, np.float32), hy)
        with pytest.raises(capi.FloodError):
            g.ensemble_products(0.2)
        g.track_max_depth(True)
        with pytest.raises(capi.FloodError):
            g.ensemble_products(0.2, (0.0,))
        with pytest.raises(capi.FloodError):
            g.ensemble_products(0.2, (1.5,))
        g.track_max_depth(False)
        with pytest.raises(capi.FloodError):
            g.max_depth(0)


def test_full_size_products_on_sampled_rows(capi):
    """2000 x 2000 cells, 96 members, one 300 s window with the maxima
    tracked, in the benchmark's launch configuration: the products on five
    sampled rows against the oracle's products of the same maxima."""
    ny = nx = 2000
    M = 96
    terr = synth.make_terrain(ny, nx, seed=1)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(1, M)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.track_max_depth(True)
        g.advance_to(300.0)
        levels = (0.1, 0.5, 0.9)
        exceed, pct = g.ensemble_products(0.01, levels)
        w = g.members()["weights"]
        # unequal weights over the same maxima (roof cells whose members
        # range from nearly dry to wet take the shifted keys)
        wu = np.linspace(1.0, 3.0, M)
        g.set_members(weights=wu / wu.sum())
        exceed_u, pct_u = g.ensemble_products(0.01, levels)
        w_u = g.members()["weights"]
        rows = np.random.default_rng(1).choice(ny, 5, replace=False)
        hm = np.array([g.max_depth(m)[rows] for m in range(M)])
    assert np.array_equal(exceed[rows], prod.exceedance(hm, w, 0.01))
    assert np.array_equal(pct[:, rows], prod.percentiles(hm, w, levels))
    assert np.array_equal(exceed_u[rows], prod.exceedance(hm, w_u, 0.01))
    assert np.array_equal(pct_u[:, rows], prod.percentiles(hm, w_u, levels))
    assert exceed.max() > 0


@pytest.mark.parametrize("M", [5, 33, 64, 96, 100, 130])
@pytest.mark.parametrize("equal", [True, False])
def test_products_every_kernel_path_bit_for_bit(capi, M, equal):
    """Every member count the products kernels distinguish (sorted in
    registers up to 96 members with any weights and up to 128 with equal
    weights, staged in shared memory beyond), with equal and with unequal
    weights set directly, on a grid whose rows end in a partial block, with
    every third member rainless (a group of maxima tied at zero in every
    cell): the maps equal the oracle's, bit for bit, for six levels (two
    passes of four)."""
    ny, nx = 12, 150
    terr = synth.make_terrain(ny, nx, seed=55)
    hy = synth.hyetograph_constant(90.0, 600.0)
    rm, sc = synth.ensemble_prior(55, M)
    rm[::3] = 0.0                                # rainless members: their maxima tie at zero
    rng = np.random.default_rng(M)
    w = np.full(M, 1.0 / M) if equal else rng.random(M) ** 3
    w = w / w.sum()
    levels = (0.05, 0.1, 0.5, 0.77, 0.9, 1.0)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.track_max_depth(True)
        g.advance_to(120.0)
        g.set_members(weights=w)
        w_dev = g.members()["weights"]
        exceed, pct = g.ensemble_products(0.003, levels)
        hm = np.array([g.max_depth(m) for m in range(M)])
    assert np.array_equal(w_dev, w)
    assert (hm == 0).sum(axis=0).min() >= (M + 2) // 3   # a tie group in every cell
    assert np.array_equal(exceed, prod.exceedance(hm, w, 0.003))
    assert np.array_equal(pct, prod.percentiles(hm, w, levels))
    assert 0 < exceed.max() <= 1.0


@pytest.mark.parametrize("M", [96, 100, 128])
def test_weighted_keys_on_crafted_maxima(capi, M):
    """Maxima set directly (the tracked maximum starts at the members'
    depths) to the cases the unequal-weights kernel treats apart: cells
    whose values span many binades (shifted keys: values one FP32 step
    apart share a place, in index order against the value order), cells
    within one binade (exact keys), exact ties, -0 beside +0, negative
    values, a threshold equal to members' values, and dyadic weights whose
    prefix sums hit the levels exactly.  The maps equal the oracle's, bit
    for bit, with unequal and with equal weights."""
    ny, nx = 4, 70
    rng = np.random.default_rng(M)
    hm = np.zeros((M, ny, nx), np.float32)
    mags = np.array([0.0, 1e-30, 1e-6, 1e-3, 0.2, 0.5, 3.0], np.float32)
    hm[:, 0] = rng.choice(mags, (M, nx)) * rng.uniform(1, 1.01, (M, nx)).astype(np.float32)
    hm[:, 1] = rng.uniform(0.2, 0.3, (M, nx)).astype(np.float32)
    hm[:, 2] = rng.choice(np.array([-0.5, -0.0, 0.0, 1e-30, 0.2], np.float32), (M, nx))
    hm[:, 3] = np.float32(0.25)
    hm[:, 3, ::3] = 0.0
    hm[: M // 2, 3, 1::3] = np.float32(0.2)
    # near ties: in rows 0 and 1 the higher index of a pair holds the smaller value
    for i in range(0, M - 1, 5):
        for r in (0, 1):
            v = hm[i + 1, r]
            hm[i, r] = np.nextafter(v, np.float32(np.inf))
    hm[1::7, 1, ::2] = np.float32(0.2)         # the threshold itself
    k = rng.integers(1, 40, M)
    k[::11] = 0                                 # weightless members
    k = k * 8192 // k.sum()
    k[np.flatnonzero(k)[: 8192 - k.sum()]] += 1
    w = k / 8192.0                              # dyadic: the prefix sums are exact
    levels = (0.05, 0.1, 0.5, 0.77, 0.9, 1.0, float(np.cumsum(w)[M // 3]), float(np.cumsum(w)[M // 2]))
    hy = synth.hyetograph_constant(0.0, 60.0)
    terr = synth.make_terrain(ny, nx, seed=56)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, np.ones(M, np.float32), np.ones(M, np.float32), hy)
        for m in range(M):
            g.set_state(m, h=hm[m])
        g.track_max_depth(True)
        got_hm = np.array([g.max_depth(m) for m in range(M)])
        g.set_members(weights=w)
        res = {th: g.ensemble_products(th, levels) for th in (0.2, 0.0)}
        g.set_members(weights=np.full(M, 1.0 / M))
        eq = g.ensemble_products(0.2, levels)
    assert np.array_equal(got_hm.view(np.uint32), hm.view(np.uint32))
    for th, (exceed, pct) in res.items():
        assert np.array_equal(exceed, prod.exceedance(hm, w, th)), th
        assert np.array_equal(pct, prod.percentiles(hm, w, levels)), th
    assert np.array_equal(eq[0], prod.exceedance(hm, np.full(M, 1.0 / M), 0.2))
    assert np.array_equal(eq[1], prod.percentiles(hm, np.full(M, 1.0 / M), levels))


@pytest.mark.parametrize("M", [1, 7, 96])
def test_products_exceedance_only_and_sixteen_levels(capi, M):
    """The call's extremes: no percentile level (the exceedance map alone,
    one pass) and the largest number of levels, sixteen (four passes of
    four), with unequal weights (equal for one member): bit for bit the
    oracle's maps."""
    ny, nx = 9, 70
    terr = synth.make_terrain(ny, nx, seed=57)
    hy = synth.hyetograph_constant(90.0, 600.0)
    rm, sc = synth.ensemble_prior(57, M)
    rng = np.random.default_rng(57 + M)
    w = rng.random(M) + 0.1
    w = w / w.sum()
    levels = tuple(np.sort(rng.uniform(0.01, 1.0, 16)))
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.track_max_depth(True)
        g.advance_to(90.0)
        g.set_members(weights=w)
        w_dev = g.members()["weights"]
        ex0, pct0 = g.ensemble_products(0.004, ())
        ex16, pct16 = g.ensemble_products(0.004, levels)
        hm = np.array([g.max_depth(m) for m in range(M)])
    want = prod.exceedance(hm, w_dev, 0.004)
    assert np.array_equal(ex0, want) and np.array_equal(ex16, want)
    assert pct0.shape[0] == 0
    assert np.array_equal(pct16, prod.percentiles(hm, w_dev, levels))


def test_weighted_keys_with_several_groups_per_warp(capi):
    """Crafted maxima (as above: values over many binades, neighbours one
    FP32 step apart, exact ties, the threshold itself) on a grid of more
    32-cell groups than the kernel has warps, so every warp sorts several
    groups while the copy of its next one lands in the same stage: the
    maps of sampled rows equal the oracle's, bit for bit."""
    ny, nx, M = 330, 300, 96
    rng = np.random.default_rng(58)
    mags = np.array([0.0, 1e-30, 1e-6, 1e-3, 0.2, 0.5, 3.0], np.float32)
    hm = rng.choice(mags, (M, ny, nx)) * rng.uniform(1, 1.01, (M, ny, nx)).astype(np.float32)
    hm[:, 1::3] = rng.uniform(0.2, 0.3, (M, ny, nx))[:, 1::3].astype(np.float32)
    for i in range(0, M - 1, 5):
        hm[i] = np.nextafter(hm[i + 1], np.float32(np.inf))
    hm[1::7, :, ::2] = np.float32(0.2)
    hm = hm.astype(np.float32)
    w = rng.random(M) ** 2 + 0.01
    w = w / w.sum()
    levels = (0.1, 0.5, 0.9)
    terr = synth.make_terrain(ny, nx, seed=58)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, np.ones(M, np.float32), np.ones(M, np.float32),
                        synth.hyetograph_constant(0.0, 60.0))
        for m in range(M):
            g.set_state(m, h=hm[m])
        g.track_max_depth(True)
        g.set_members(weights=w)
        w_dev = g.members()["weights"]
        exceed, pct = g.ensemble_products(0.2, levels)
    rows = np.random.default_rng(59).choice(ny, 12, replace=False)
    sub = hm[:, rows]
    assert np.array_equal(exceed[rows], prod.exceedance(sub, w_dev, 0.2))
    assert np.array_equal(pct[:, rows], prod.percentiles(sub, w_dev, levels))
