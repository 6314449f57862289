"""GPU inflow hydrograph boundary: a discharge series entering through a
segment of the west edge, against the FP64 oracle, bit for bit across
engines and launch shapes, exact storage in a closed box, refusals."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import compare, oracle_params, require_gpu

pytestmark = pytest.mark.gpu

SERIES = np.array([4.0, 6.0, 2.0], np.float32)


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _run(capi, terr, hy, rm, sc, r0, r1, t_end, engine=None, shape=None, params=None):
    M = len(rm)
    with capi.Grid(terr.z, terr.n, params) as g:
        g.set_inflow(r0, r1, SERIES)
        g.ensemble_init(M, rm, sc, hy)
        if engine is not None:
            g.set_engine(engine)
        if shape is not None:
            g.set_launch(*shape)
        g.advance_to(t_end)
        g.sync()
        return [g.get_state(m) for m in range(M)], g.members(), g.volumes(), g.inflow_volume()


def test_inflow_follows_the_oracle(capi):
    ny, nx = 48, 80
    terr = synth.make_terrain(ny, nx, seed=92, building_frac=0.02)
    hy = synth.hyetograph_constant(30.0, 900.0)
    rm, sc = synth.ensemble_prior(92, 2)
    p = capi.Params.default()
    states, mem, vol, inflow = _run(capi, terr, hy, rm, sc, 10, 30, 900.0, params=p)
    for m in range(2):
        op = oracle_params(p, ny, nx)
        op.inflow = SERIES.astype(np.float64)
        op.inflow_r0, op.inflow_r1 = 10, 30
        mo = oracle.Member.dry(ny, nx)
        oracle.advance(op, terr.z, terr.n, float(sc[m]), float(rm[m]), hy, mo, t_end=900.0)
        compare(states[m][0], mo.h, 1e-3)
        assert abs(inflow[m] - mo.inflow) <= 1e-6 * mo.inflow
        V = vol["storage"][m]
        bal = V - (vol["rain"][m] + inflow[m] - vol["outflow"][m] + vol["clamp"][m])
        assert abs(bal) <= 1e-5 * (vol["rain"][m] + inflow[m])
        assert np.all(states[m][1][10:30, 0] > 0)  # the inflow rows' first links carry water east


@pytest.mark.parametrize("case", [(0, (16, 4)), (1, (7, 1)), (1, (64, 4)), (0, (5, 1))])
def test_inflow_engines_and_shapes_bitwise(capi, case):
    terr = synth.make_terrain(45, 150, seed=93)
    hy = synth.hyetograph_constant(60.0, 600.0)
    rm, sc = synth.ensemble_prior(93, 5)
    ref = _run(capi, terr, hy, rm, sc, 9, 37, 400.0, engine=1)
    got = _run(capi, terr, hy, rm, sc, 9, 37, 400.0, engine=case[0], shape=case[1])
    for m in range(5):
        for k in range(3):
            assert np.array_equal(got[0][m][k], ref[0][m][k])
    assert np.array_equal(got[3], ref[3])


def test_closed_flat_box_stores_the_inflow(capi):
    ny, nx = 20, 40
    z = np.zeros((ny, nx), np.float32)
    n = np.full((ny, nx), 0.04, np.float32)
    p = capi.Params.default(east_outflow=0, dt_cap=0.5)
    with capi.Grid(z, n, p) as g:
        g.set_inflow(5, 15, SERIES)
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), np.zeros(3, np.float32))
        g.advance_to(900.0)
        V = g.volumes()["storage"][0]
        vin = g.inflow_volume()[0]
    want = 300.0 * float(SERIES.astype(np.float64).sum())
    assert abs(vin - want) <= 1e-6 * want
    assert abs(V - want) <= 1e-5 * want


def test_inflow_refusals_and_removal(capi):
    terr = synth.make_terrain(20, 30, seed=94)
    hy = synth.hyetograph_constant(50.0, 300.0)
    with capi.Grid(terr.z, terr.n) as g:
        for r0, r1 in [(-1, 5), (5, 21), (7, 7)]:
            with pytest.raises(capi.FloodError):
                g.set_inflow(r0, r1, SERIES)
        with pytest.raises(capi.FloodError):
            g.set_inflow(2, 8, np.array([1.0, -2.0], np.float32))
        g.set_inflow(2, 8, SERIES)
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), hy)
        g.set_inflow(0, 1, np.zeros(0, np.float32))  # removed: the west edge is a wall again
        g.advance_to(120.0)
        assert g.inflow_volume()[0] == 0.0


def _wet_inflow_case(ny=40, nx=56, M=2, seed=95):
    terr = synth.make_terrain(ny, nx, seed=seed, building_frac=0.0)
    zmax = float(terr.z.max())
    h0 = np.maximum(0.15 + 0.4 * (zmax - terr.z) / max(zmax, 1e-6), 0.15).astype(np.float32)
    rng = np.random.default_rng(seed)
    rm = rng.uniform(0.8, 1.3, M).astype(np.float32)
    sc = rng.uniform(0.8, 1.2, M).astype(np.float32)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    cells = np.array([12 * nx + 1, 20 * nx + 4, 30 * nx + 30, 5 * nx + 50], np.int32)
    ns, sdt = 6, 30.0
    d = (h0.ravel()[cells][None, :] + rng.normal(0, 0.02, (ns, 4))).astype(np.float64)
    return terr, h0, rm, sc, hy, cells, d, sdt


def test_adjoint_with_inflow_matches_the_oracle_adjoint(capi):
    """The reverse mode across an inflow boundary (the flux is prescribed, so
    it only shifts the depths every other derivative is taken at) against
    the FP64 oracle's adjoint with the same inflow."""
    terr, h0, rm, sc, hy, cells, d, sdt = _wet_inflow_case()
    ny, nx = terr.z.shape
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.set_inflow(8, 24, SERIES)
        g.ensemble_init(len(rm), rm, sc, hy, h0=h0)
        out = g.adjoint(cells, d, sdt)
    op = oracle_params(p, ny, nx)
    op.inflow = SERIES.astype(np.float64)
    op.inflow_r0, op.inflow_r1 = 8, 24
    gn_sum = np.zeros(terr.z.shape)
    for m in range(len(rm)):
        r = oracle.loss_and_grad(op, terr.z, terr.n, float(sc[m]), float(rm[m]), hy, h0, sdt, d,
                                 cells)
        assert abs(out["loss"][m] - r["loss"]) <= 1e-4 * r["loss"]
        assert abs(out["grad_rain"][m] - r["grad_rain"]) <= 2e-3 * abs(r["grad_rain"])
        assert abs(out["grad_scale"][m] - r["grad_scale"]) <= 2e-3 * abs(r["grad_scale"])
        gh = out["grad_h0"][m]
        assert np.max(np.abs(gh - r["grad_h0"])) <= 2e-3 * np.max(np.abs(r["grad_h0"]))
        gn_sum += r["grad_n"]
    assert np.max(np.abs(out["grad_n"] - gn_sum)) <= 2e-3 * np.max(np.abs(gn_sum))


@pytest.mark.parametrize("M", [1, 5])
def test_adjoint_with_inflow_engines_bitwise(capi, M):
    """Direct-load and TMA-staged replay and reverse stencil with an inflow
    boundary: the same gradients, bit for bit."""
    terr, h0, rm, sc, hy, cells, d, sdt = _wet_inflow_case(ny=45, nx=150, M=M, seed=96)
    res = []
    for engine in (0, 1):
        with capi.Grid(terr.z, terr.n) as g:
            g.set_inflow(5, 30, SERIES)
            g.ensemble_init(M, rm, sc, hy, h0=h0)
            g.set_engine(engine)
            g.set_launch(16, 4 if M >= 4 else 1)
            res.append(g.adjoint(cells, d, sdt, ckpt_every=5))
    for key in ("loss", "grad_rain", "grad_scale", "grad_n", "grad_h0"):
        assert np.array_equal(res[0][key], res[1][key]), key
