"""Pins of the FP64 oracle's scheme (Eq. 1-5, Section 2.1) against what the
paper and the mathematics fix: the paper's worked time-step numbers
(Section 4.1), Manning normal flow as the fixed point of Eq. 2, the shallow
water gravity-wave speed sqrt(g h) (seiche period), lake at rest, uniform
rain, exact volume balance, x/y transposition symmetry and the no-climb
property of Eq. 3.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_dt_matches_section_4_1_numbers():
    """Section 4.1: with k = 0.54, 3 m cells and h_max = 4.2 m, Eq. 4 allows
    just over the 0.25 s the paper used (0.54*3/sqrt(9.81*4.2) = 0.2524 s)."""
    g = json.load(open(os.path.join(GOLD, "dt_section_4_1.json")))
    p = oracle.Params(ny=1, nx=1, dx=g["dx"], g=g["g"], alpha=g["k"], dt_cap=1e9, rain_block=1e9)
    dt, tn = oracle.dt(p, g["h_max"], 0.0)
    assert dt >= g["dt_used_by_paper"]
    assert abs(dt - g["dt_max_rounded"]) < 5e-5
    assert tn == dt


def test_dt_floor_cap_fixed_and_event_clipping():
    p = oracle.Params(ny=1, nx=1)
    # dry domain: floor makes Eq. 4 huge, the cap wins
    assert oracle.dt(p, 0.0, 0.0)[0] == p.dt_cap
    # deep water: Eq. 4 wins, dt ~ 1/sqrt(h)
    d1, _ = oracle.dt(p, 4.0, 0.0)
    d2, _ = oracle.dt(p, 16.0, 0.0)
    assert abs(d1 / d2 - 2.0) < 1e-14
    # lands exactly on the rain-block edge and on t_end
    dt, tn = oracle.dt(p, 0.0, 299.75, -1.0)
    assert tn == 300.0 and abs(dt - 0.25) < 1e-12
    dt, tn = oracle.dt(p, 0.0, 10.0, 10.4)
    assert tn == 10.4
    # fixed-step mode (the paper's 0.25 s, Section 4.1)
    pf = oracle.Params(ny=1, nx=1, dt_fixed=0.25)
    assert oracle.dt(pf, 100.0, 0.0)[0] == 0.25


def test_two_cell_hand_steps():
    g = json.load(open(os.path.join(GOLD, "two_cell_steps.json")))
    p = oracle.Params(ny=1, nx=2, dx=g["dx"], g=g["g"], east_outflow=0)
    m = oracle.Member.dry(1, 2, np.array([g["h0"]]))
    z = np.zeros((1, 2)); n = np.full((1, 2), g["n"])
    for s in g["steps"]:
        oracle.step(p, z, n, 1.0, 0.0, g["dt"], m)
        assert abs(m.qx[0, 1] - s["q"]) < g["tolerance"]
        assert np.allclose(m.h[0], s["h"], rtol=0, atol=g["tolerance"])
        assert m.qx[0, 0] == 0.0 and m.qx[0, 2] == 0.0


@pytest.mark.parametrize("dt", [0.05, 0.3, 2.0, 10.0])
def test_manning_normal_flow_is_fixed_point_of_eq2(dt):
    """On a plane of slope S0 with uniform depth h, the Manning discharge
    q = h^(5/3) S0^(1/2) / n solves q = (q + g h dt S0)/(1 + g n^2 q dt/h^(7/3))
    for every dt: Eq. 2 must leave it unchanged on interior links, and the
    free-outflow edge (a normal-depth boundary continuing the bed slope) must
    pass the same uniform flow."""
    ny, nx, dx, S0, h0, nman = 3, 24, 3.0, 0.004, 0.4, 0.035
    p = oracle.Params(ny=ny, nx=nx, dx=dx, limiter=0, east_outflow=1, edge_slope=S0)
    c = np.arange(nx)
    z = np.broadcast_to(S0 * dx * (nx - 1 - c), (ny, nx)).copy()
    n = np.full((ny, nx), nman)
    m = oracle.Member.dry(ny, nx, np.full((ny, nx), h0))
    qn = h0 ** (5.0 / 3.0) * math.sqrt(S0) / nman
    m.qx[:, 1:] = qn
    oracle.step(p, z, n, 1.0, 0.0, dt, m)
    assert np.allclose(m.qx[:, 1:], qn, rtol=1e-12, atol=0)
    assert np.all(m.qy == 0.0)
    # a scaled Manning field (per-member scale) is the same as a larger n
    m2 = oracle.Member.dry(ny, nx, np.full((ny, nx), h0))
    m2.qx[:, 1:] = qn / 1.3
    oracle.step(p, z, n, 1.3, 0.0, dt, m2)
    assert np.allclose(m2.qx[:, 1:], qn / 1.3, rtol=1e-12, atol=0)


def test_seiche_period_is_2L_over_sqrt_gH():
    """Frictionless small-amplitude standing wave in a closed basin of length
    L: the first mode has period T = 2 L / sqrt(g H) (linear shallow-water
    theory).  After T/2 the cosine mode is inverted, after T restored."""
    nx, dx, H, a = 120, 3.0, 1.0, 1e-3
    L = nx * dx
    T = 2 * L / math.sqrt(9.81 * H)
    nsteps = 1200
    dt = T / nsteps
    p = oracle.Params(ny=1, nx=nx, dx=dx, dt_fixed=dt, east_outflow=0, rain_block=1e9)
    xc = (np.arange(nx) + 0.5) / nx
    mode = np.cos(np.pi * xc)
    m = oracle.Member.dry(1, nx, (H + a * mode)[None, :])
    z = np.zeros((1, nx)); n = np.zeros((1, nx))

    def amp():
        return 2.0 / nx * float(((m.h[0] - H) * mode).sum()) / a

    # at T/4 the mode passes through zero: |amp| ~ (pi/2) * relative period error
    for _ in range(nsteps // 4):
        oracle.step(p, z, n, 1.0, 0.0, dt, m)
    assert abs(amp()) < 3e-3
    for _ in range(nsteps // 4):
        oracle.step(p, z, n, 1.0, 0.0, dt, m)
    assert abs(amp() + 1.0) < 1e-3
    for _ in range(nsteps // 2):
        oracle.step(p, z, n, 1.0, 0.0, dt, m)
    assert abs(amp() - 1.0) < 1e-3


def test_lake_at_rest_over_bumpy_bed():
    """Flat water surface over an uneven bed with dry islands: every link has
    zero slope or zero flow depth, so nothing moves, exactly."""
    rng = np.random.default_rng(7)
    ny, nx = 20, 24
    z = rng.integers(0, 2600, (ny, nx)) * 2.0 ** -10       # dyadic, exact in FP32/FP64
    eta = 2.0
    h = np.maximum(eta - z, 0.0)
    p = oracle.Params(ny=ny, nx=nx, east_outflow=0)
    n = np.full((ny, nx), 0.05)
    m = oracle.Member.dry(ny, nx, h)
    oracle.advance(p, z, n, 1.0, 1.0, np.zeros(1), m, max_steps=200)
    assert (z > eta).any() and (h > 0.5).any()
    assert np.array_equal(m.h, h)
    assert not m.qx.any() and not m.qy.any()


def test_uniform_rain_on_flat_closed_box():
    ny, nx = 9, 11
    p = oracle.Params(ny=ny, nx=nx, east_outflow=0, dt_cap=0.37)
    z = np.full((ny, nx), 1.25); n = np.full((ny, nx), 0.05)
    hy = synth.hyetograph_constant(50.0, 600.0).astype(np.float64)
    m = oracle.Member.dry(ny, nx)
    dts = oracle.advance(p, z, n, 1.0, 1.2, hy, m, t_end=600.0, log_dt=True)
    expect = 0.0
    for d in dts:
        expect = expect + d * (float(hy[0]) * 1.2)
    assert m.t == 600.0
    assert np.all(m.h == expect)
    assert abs(expect - float(hy[0]) * 1.2 * 600.0) < 1e-12 * expect
    assert abs(float(hy[0]) - 50.0 / 3.6e6) < 1e-6 * float(hy[0])
    assert not m.qx.any() and not m.qy.any()


def _dem(ny, nx, seed):
    t = synth.make_terrain(ny, nx, seed)
    return t.z.astype(np.float64), t.n.astype(np.float64)


def test_volume_balance_exact_to_1e12():
    """Eq. 5 only moves volume between cells: storage change = rain - outflow
    (+ clamp), to 1e-12 of the rain volume."""
    ny, nx = 48, 64
    z, n = _dem(ny, nx, 11)
    p = oracle.Params(ny=ny, nx=nx)
    hy = np.array([200.0, 80.0]) / 3.6e6
    m = oracle.Member.dry(ny, nx)
    oracle.advance(p, z, n, 1.1, 1.0, hy, m, t_end=450.0)
    V = oracle.storage(m.h, p.dx)
    assert m.outflow > 0
    assert abs(V - (m.rain - m.outflow + m.clamp)) <= 1e-12 * m.rain
    assert m.clamp <= 1e-12 * m.rain
    assert m.h.min() >= 0.0


def test_transposition_symmetry():
    """Swapping x and y (rows <-> columns, east <-> south outflow) transposes
    the solution."""
    ny, nx = 30, 44
    z, n = _dem(ny, nx, 5)
    hy = np.array([120.0]) / 3.6e6
    p = oracle.Params(ny=ny, nx=nx, east_outflow=1, south_outflow=0)
    pt = oracle.Params(ny=nx, nx=ny, east_outflow=0, south_outflow=1)
    a = oracle.Member.dry(ny, nx)
    b = oracle.Member.dry(nx, ny)
    oracle.advance(p, z, n, 0.9, 1.0, hy, a, t_end=200.0)
    oracle.advance(pt, z.T.copy(), n.T.copy(), 0.9, 1.0, hy, b, t_end=200.0)
    assert a.steps == b.steps
    assert np.allclose(a.h, b.h.T, rtol=0, atol=1e-13)
    assert np.allclose(a.qx, b.qy.T, rtol=0, atol=1e-13)
    assert abs(a.outflow - b.outflow) <= 1e-12 * a.rain


def test_no_flow_over_a_dry_wall_eq3():
    """Eq. 3: a pond below the crest of a dry neighbour has zero flow depth on
    the shared link, so (limiter off) no water is drawn out of the dry cell."""
    p = oracle.Params(ny=1, nx=3, limiter=0, east_outflow=0)
    z = np.array([[0.0, 5.0, 0.0]]); n = np.full((1, 3), 0.05)
    m = oracle.Member.dry(1, 3, np.array([[1.0, 0.0, 0.3]]))
    for _ in range(20):
        oracle.step(p, z, n, 1.0, 0.0, 0.5, m)
    assert m.clamp == 0.0
    assert np.array_equal(m.h, [[1.0, 0.0, 0.3]])
    # water above the crest does spill over, from the pond side
    m = oracle.Member.dry(1, 3, np.array([[5.5, 0.0, 0.0]]))
    oracle.step(p, z, n, 1.0, 0.0, 0.1, m)
    assert m.qx[0, 1] > 0 and m.h[0, 1] > 0


def test_shallow_sheet_below_h_eps_does_not_move():
    """The optional wet/dry threshold: links with flow depth <= h_eps carry
    nothing."""
    ny, nx = 4, 10
    p = oracle.Params(ny=ny, nx=nx, h_eps=1e-3)
    z = np.broadcast_to(0.05 * (nx - 1 - np.arange(nx)), (ny, nx)).copy()
    m = oracle.Member.dry(ny, nx, np.full((ny, nx), 0.9e-3))
    oracle.advance(p, z, np.full((ny, nx), 0.03), 1.0, 1.0, np.zeros(1), m, max_steps=50)
    assert not m.qx.any() and np.all(m.h == 0.9e-3)


def test_free_outflow_passes_outward_only():
    ny, nx = 3, 6
    p = oracle.Params(ny=ny, nx=nx)
    z = np.zeros((ny, nx)); n = np.full((ny, nx), 0.03)
    m = oracle.Member.dry(ny, nx, np.full((ny, nx), 0.2))
    V0 = oracle.storage(m.h, p.dx)
    last = V0
    for _ in range(60):
        oracle.step(p, z, n, 1.0, 0.0, 0.5, m)
        assert np.all(m.qx[:, nx] >= 0.0)
        V = oracle.storage(m.h, p.dx)
        assert V <= last + 1e-15
        last = V
    assert abs(V0 - last - m.outflow) < 1e-12 * V0
    assert m.outflow > 0.05 * V0
    # a dry edge cell draws nothing from the ghost
    m = oracle.Member.dry(ny, nx)
    oracle.step(p, z, n, 1.0, 0.0, 0.5, m)
    assert not m.qx.any()


def test_positivity_with_limiter_on_urban_dem():
    ny, nx = 40, 40
    z, n = _dem(ny, nx, 3)
    p = oracle.Params(ny=ny, nx=nx)
    hy = np.array([400.0, 400.0]) / 3.6e6
    m = oracle.Member.dry(ny, nx)
    oracle.advance(p, z, n, 0.6, 1.0, hy, m, t_end=600.0)
    assert m.h.min() >= 0.0
    assert m.clamp <= 1e-12 * m.rain
