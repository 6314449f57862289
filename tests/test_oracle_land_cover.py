"""Pins of the oracle's land cover (Section 4.1): the runoff coefficient
scales the rain that stays on the surface, the drainage rate removes water
while there is any, and cells outside the domain (a wall class: bed raised
out of reach, no rain) stay dry and pass no flow.  Closed forms on a flat
closed box, the volume balance with the drained volume, and the wall."""
import numpy as np

import oracle
from paper_2302_08341_gb300 import synth

WALL_Z = 1.0e6


def _flat_box(ny=9, nx=13, rc=1.0, drain=0.0):
    p = oracle.Params(ny=ny, nx=nx, east_outflow=0, dt_cap=0.5)
    p.rc = np.full((ny, nx), rc)
    p.drain = np.full((ny, nx), drain)
    return p, np.zeros((ny, nx)), np.full((ny, nx), 0.05)


def test_flat_box_rain_above_drainage_closed_form():
    """Uniform class, rain c*r above the drainage d: no flow, h = (c r - d) T."""
    r, c, d, T = 60.0 / 3.6e6, 0.9, 12.0 / 3.6e6, 900.0
    p, z, n = _flat_box(rc=c, drain=d)
    hy = np.full(4, r)
    m = oracle.Member.dry(p.ny, p.nx)
    oracle.advance(p, z, n, 1.0, 1.0, hy, m, t_end=T)
    want = (c * r - d) * T
    assert np.allclose(m.h, want, rtol=1e-12, atol=0)
    assert np.all(m.qx == 0) and np.all(m.qy == 0)
    A = p.dx * p.dx * p.ny * p.nx
    assert np.isclose(m.rain, c * r * T * A, rtol=1e-12)
    assert np.isclose(m.drained, d * T * A, rtol=1e-12)


def test_flat_box_drainage_above_rain_takes_all():
    """Drainage faster than the rain: the surface stays dry and every drop
    that stays on the surface is drained (never more)."""
    r, c, d, T = 10.0 / 3.6e6, 0.9, 12.0 / 3.6e6, 600.0
    p, z, n = _flat_box(rc=c, drain=d)
    m = oracle.Member.dry(p.ny, p.nx)
    oracle.advance(p, z, n, 1.0, 1.0, np.full(3, r), m, t_end=T)
    assert np.all(m.h == 0.0)
    assert np.isclose(m.drained, m.rain, rtol=1e-12) and m.clamp == 0.0
    assert np.isclose(m.rain, c * r * T * p.dx * p.dx * p.ny * p.nx, rtol=1e-12)


def test_volume_balance_with_land_cover_exact_to_1e12():
    terr = synth.make_terrain(40, 60, seed=7)
    rng = np.random.default_rng(7)
    cls = rng.integers(0, 3, terr.z.shape)
    p = oracle.Params(ny=40, nx=60)
    p.rc = np.array([0.9, 1.0, 1.0])[cls].astype(np.float64)
    p.drain = np.array([0.0, 0.0, 12.0 / 3.6e6])[cls].astype(np.float64)
    hy = synth.hyetograph_constant(80.0, 900.0)
    m = oracle.Member.dry(40, 60)
    oracle.advance(p, terr.z, terr.n, 1.0, 1.0, hy, m, t_end=900.0)
    V = oracle.storage(m.h, p.dx)
    assert m.drained > 0 and m.outflow >= 0
    assert abs(V - (m.rain - m.outflow + m.clamp - m.drained)) <= 1e-12 * m.rain
    assert m.h.min() >= 0.0


def test_wall_cells_stay_dry_and_pass_no_flow():
    """A block of wall cells (bed out of reach, no rain) inside a rainy,
    sloping domain: the block stays dry and no link into it carries flow."""
    ny, nx = 20, 30
    terr = synth.make_terrain(ny, nx, seed=8, building_frac=0.0)
    z = terr.z.astype(np.float64).copy()
    wall = np.zeros((ny, nx), bool)
    wall[6:12, 10:17] = True
    wall[:, -1] = False
    z[wall] = WALL_Z
    p = oracle.Params(ny=ny, nx=nx)
    p.rc = np.where(wall, 0.0, 1.0)
    p.drain = np.zeros((ny, nx))
    m = oracle.Member.dry(ny, nx)
    oracle.advance(p, z, terr.n, 1.0, 1.0, synth.hyetograph_constant(100.0, 600.0), m, t_end=600.0)
    assert np.all(m.h[wall] == 0.0)
    assert m.h[~wall].min() > 0.0
    # x links with a wall cell on either side (oracle link c lies between c-1 and c)
    wl = np.zeros_like(m.qx, bool)
    wl[:, 1:] |= wall
    wl[:, :-1] |= wall
    assert np.all(m.qx[wl] == 0.0)
    wy = np.zeros_like(m.qy, bool)
    wy[1:, :] |= wall
    wy[:-1, :] |= wall
    assert np.all(m.qy[wy] == 0.0)
    assert abs(oracle.storage(m.h, p.dx) - (m.rain - m.outflow + m.clamp)) <= 1e-12 * m.rain
