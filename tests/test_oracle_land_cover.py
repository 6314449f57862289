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


def test_adjoint_with_land_cover_matches_central_differences():
    """The reverse mode with land cover (class roughness as the n field, the
    runoff coefficient on the rain, drainage that leaves water behind) in
    the fully wet regime with a fixed step schedule: central differences of
    the forward oracle."""
    ny, nx = 10, 14
    rng = np.random.default_rng(9)
    yy, xx = np.mgrid[0:ny, 0:nx]
    z = 0.004 * 3.0 * (nx - 1 - xx) + 0.05 * np.sin(0.7 * yy) * np.cos(0.5 * xx)
    cls = rng.integers(0, 3, (ny, nx))
    n = np.array([0.05, 0.03, 0.035])[cls]
    h0 = 0.35 + 0.1 * np.exp(-((yy - ny / 2) ** 2 + (xx - nx / 3) ** 2) / 8.0)
    p = oracle.Params(ny=ny, nx=nx, dt_cap=0.5, dt_fixed=0.5)
    p.rc = np.array([0.9, 1.0, 1.0])[cls].astype(np.float64)
    p.drain = np.array([0.0, 0.0, 20.0 / 3.6e6])[cls].astype(np.float64)
    hy = np.array([40.0, 10.0]) / 3.6e6
    cells = np.array([3 * nx + 4, 6 * nx + 9, 8 * nx + 12], np.int32)
    d = np.array([[0.40, 0.33, 0.30], [0.38, 0.35, 0.31], [0.36, 0.34, 0.33]])

    def loss(n_, scale, rm, h0_):
        return oracle.loss_and_grad(p, z, n_, scale, rm, hy, h0_, 20.0, d, cells)["loss"]

    res = oracle.loss_and_grad(p, z, n, 1.1, 1.3, hy, h0, 20.0, d, cells)
    assert np.isfinite(res["loss"]) and res["steps"] == 120
    eps = 1e-6
    fd = (loss(n, 1.1, 1.3 + eps, h0) - loss(n, 1.1, 1.3 - eps, h0)) / (2 * eps)
    assert abs(fd - res["grad_rain"]) <= 1e-6 * abs(fd) + 1e-12
    fd = (loss(n, 1.1 + eps, 1.3, h0) - loss(n, 1.1 - eps, 1.3, h0)) / (2 * eps)
    assert abs(fd - res["grad_scale"]) <= 1e-5 * abs(fd) + 1e-12
    drain = p.drain.copy()
    lk = []
    for k in (1.0 + eps, 1.0 - eps):
        p.drain = np.ascontiguousarray(drain * k)
        lk.append(loss(n, 1.1, 1.3, h0))
    p.drain = drain
    fd = (lk[0] - lk[1]) / (2 * eps)
    assert res["grad_drain"] != 0.0
    assert abs(fd - res["grad_drain"]) <= 1e-5 * abs(fd) + 1e-12
    # a step of 1e-6 in one cell's depth can cross a switch of max(eta) on a
    # link (the derivative there is one-sided), 1e-7 stays clear of it
    for i in rng.choice(ny * nx, 6, replace=False):
        for name, arr in (("grad_n", n), ("grad_h0", h0)):
            e = 1e-7
            ap = arr.copy(); ap.flat[i] += e
            am = arr.copy(); am.flat[i] -= e
            if name == "grad_n":
                fd = (loss(ap, 1.1, 1.3, h0) - loss(am, 1.1, 1.3, h0)) / (2 * e)
            else:
                fd = (loss(n, 1.1, 1.3, ap) - loss(n, 1.1, 1.3, am)) / (2 * e)
            g = res[name].flat[i]
            assert abs(fd - g) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(res[name]).max()), (name, i, fd, g)


def test_adjoint_drainage_that_takes_everything_passes_nothing():
    """Closed form: on a flat closed box whose drainage per step exceeds the
    water present, every cell is emptied at the first step, so the observed
    depths (0) depend neither on the initial depth nor on the rain
    multiplier; without the drained branch the gradients would be 2 (0 - d)
    per observation."""
    p, z, n = _flat_box(ny=6, nx=8, rc=1.0, drain=3600.0 / 3.6e6)   # 1 m/h ≫ the 1 mm present
    p.dt_fixed = 0.5
    h0 = np.full(z.shape, 1e-3)
    hy = np.array([10.0]) / 3.6e6
    cells = np.array([9, 20], np.int32)
    d = np.array([[0.01, 0.02]])
    res = oracle.loss_and_grad(p, z, n, 1.0, 1.0, hy, h0, 5.0, d, cells)
    assert np.isclose(res["loss"], 0.01 ** 2 + 0.02 ** 2, rtol=1e-12)
    assert np.all(res["grad_h0"] == 0.0) and res["grad_rain"] == 0.0


def test_adjoint_flat_box_rain_above_drainage_closed_form():
    """Closed form: on a flat closed box of one class the depth is
    h(t) = (c r m - kappa d) t everywhere, so with e = h(t_s) - d_s the
    gradients are dL/dm = sum 2 e c r t_s and dL/dkappa = -sum 2 e d t_s."""
    r, c, dr, m = 60.0 / 3.6e6, 0.9, 12.0 / 3.6e6, 1.2
    p, z, n = _flat_box(rc=c, drain=dr)
    hy = np.array([r])
    cells = np.array([14, 60, 100], np.int32)
    sdt, ns = 30.0, 4
    ts = sdt * np.arange(1, ns + 1)
    obs = np.array([[0.0004, 0.0009, 0.0002]] * ns) * np.arange(1, ns + 1)[:, None]
    res = oracle.loss_and_grad(p, z, n, 1.0, m, hy, 0.0, sdt, obs, cells)
    e = (c * r * m - dr) * ts[:, None] - obs
    assert np.isclose(res["loss"], (e ** 2).sum(), rtol=1e-10)
    assert np.isclose(res["grad_rain"], (2 * e * c * r * ts[:, None]).sum(), rtol=1e-9)
    assert np.isclose(res["grad_drain"], -(2 * e * dr * ts[:, None]).sum(), rtol=1e-9)
