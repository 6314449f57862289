"""Pins of the oracle's inflow hydrograph boundary (a discharge series
entering through a segment of the west edge, spread evenly over its links):
exact stored volume in a closed flat box for a constant and for a
piecewise-constant series, and the volume balance with rain, inflow and
outflow over an urban DEM to 1e-12.  CPU only."""
import numpy as np

import oracle
from paper_2302_08341_gb300 import synth


def _box(ny=10, nx=16, r0=3, r1=8, series=(2.0,)):
    p = oracle.Params(ny=ny, nx=nx, east_outflow=0, dt_cap=0.5)
    p.inflow = np.asarray(series, np.float64)
    p.inflow_r0, p.inflow_r1 = r0, r1
    return p, np.zeros((ny, nx)), np.full((ny, nx), 0.04)


def test_closed_box_stores_the_inflow_exactly():
    p, z, n = _box(series=(2.0,) * 3)
    m = oracle.Member.dry(p.ny, p.nx)
    oracle.advance(p, z, n, 1.0, 1.0, np.zeros(3), m, t_end=600.0)
    assert np.isclose(oracle.storage(m.h, p.dx), 2.0 * 600.0, rtol=1e-12)
    assert np.isclose(m.inflow, 2.0 * 600.0, rtol=1e-12)
    assert m.qx[p.inflow_r0, 0] > 0 and m.qx[0, 0] == 0.0 and m.qx[p.ny - 1, 0] == 0.0
    # the flux per unit width on each inflow link is Q / (dx * rows)
    assert np.allclose(m.qx[p.inflow_r0:p.inflow_r1, 0], 2.0 / (p.dx * 5), rtol=1e-15)


def test_piecewise_series_lands_on_block_edges():
    p, z, n = _box(series=(2.0, 0.5, 0.0))
    m = oracle.Member.dry(p.ny, p.nx)
    oracle.advance(p, z, n, 1.0, 1.0, np.zeros(3), m, t_end=900.0)
    assert np.isclose(oracle.storage(m.h, p.dx), 2.0 * 300.0 + 0.5 * 300.0, rtol=1e-12)


def test_volume_balance_with_inflow_and_rain_to_1e12():
    terr = synth.make_terrain(40, 60, seed=91)
    p = oracle.Params(ny=40, nx=60)
    p.inflow = np.array([5.0, 8.0, 3.0])
    p.inflow_r0, p.inflow_r1 = 12, 25
    hy = synth.hyetograph_constant(40.0, 900.0)
    m = oracle.Member.dry(40, 60)
    oracle.advance(p, terr.z, terr.n, 1.0, 1.0, hy, m, t_end=900.0)
    V = oracle.storage(m.h, p.dx)
    assert m.inflow > 0 and m.outflow > 0
    assert abs(V - (m.rain + m.inflow - m.outflow + m.clamp)) <= 1e-12 * (m.rain + m.inflow)


def test_adjoint_with_inflow_matches_central_differences():
    """The reverse mode across an inflow boundary: the inflow flux is
    prescribed (no derivative of its own) but raises the depths downstream,
    so every other derivative moves; central differences of the forward
    oracle agree (fully wet, fixed step schedule)."""
    ny, nx = 10, 14
    rng = np.random.default_rng(5)
    yy, xx = np.mgrid[0:ny, 0:nx]
    z = 0.004 * 3.0 * (nx - 1 - xx) + 0.05 * np.sin(0.7 * yy) * np.cos(0.5 * xx)
    n = 0.03 + 0.02 * rng.random((ny, nx))
    h0 = 0.35 + 0.1 * np.exp(-((yy - ny / 2) ** 2 + (xx - nx / 3) ** 2) / 8.0)
    hy = np.array([40.0, 10.0]) / 3.6e6
    cells = np.array([3 * nx + 2, 6 * nx + 5, 8 * nx + 12], np.int32)
    d = np.array([[0.40, 0.33, 0.30], [0.38, 0.35, 0.31], [0.36, 0.34, 0.33]])

    def params(inflow):
        p = oracle.Params(ny=ny, nx=nx, dt_cap=0.5, dt_fixed=0.5)
        if inflow:
            p.inflow = np.array([1.5, 0.5])
            p.inflow_r0, p.inflow_r1 = 2, 7
        return p

    p = params(True)

    def loss(n_, scale, rm, h0_):
        return oracle.loss_and_grad(p, z, n_, scale, rm, hy, h0_, 20.0, d, cells)["loss"]

    res = oracle.loss_and_grad(p, z, n, 1.1, 1.3, hy, h0, 20.0, d, cells)
    plain = oracle.loss_and_grad(params(False), z, n, 1.1, 1.3, hy, h0, 20.0, d, cells)
    assert np.isfinite(res["loss"]) and res["steps"] == 120
    assert abs(res["grad_rain"] - plain["grad_rain"]) > 1e-6 * abs(plain["grad_rain"])
    eps = 1e-6
    fd = (loss(n, 1.1, 1.3 + eps, h0) - loss(n, 1.1, 1.3 - eps, h0)) / (2 * eps)
    assert abs(fd - res["grad_rain"]) <= 1e-6 * abs(fd) + 1e-12
    fd = (loss(n, 1.1 + eps, 1.3, h0) - loss(n, 1.1 - eps, 1.3, h0)) / (2 * eps)
    assert abs(fd - res["grad_scale"]) <= 1e-5 * abs(fd) + 1e-12
    for i in [2 * nx + 0, 4 * nx + 1, 5 * nx + 3, 7 * nx + 8]:   # next to the inflow and beyond
        for name, arr in (("grad_n", n), ("grad_h0", h0)):
            e = eps * max(1.0, abs(arr.flat[i]))
            ap = arr.copy(); ap.flat[i] += e
            am = arr.copy(); am.flat[i] -= e
            if name == "grad_n":
                fd = (loss(ap, 1.1, 1.3, h0) - loss(am, 1.1, 1.3, h0)) / (2 * e)
            else:
                fd = (loss(n, 1.1, 1.3, ap) - loss(n, 1.1, 1.3, am)) / (2 * e)
            g = res[name].flat[i]
            assert abs(fd - g) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(res[name]).max()), (name, i, fd, g)
