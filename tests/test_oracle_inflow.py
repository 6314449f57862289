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
