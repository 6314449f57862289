"""Pins of the oracle's section discharge (streamflow gauges, Section 4.4's
stream gauges): the discharges through the four sides of any box of cells
close the box's water balance over a step (Eq. 5 with Eq. 1), and uniform
Manning flow through a section of a tilted plane is the closed-form normal
discharge.  CPU only."""
import numpy as np

import oracle
from paper_2302_08341_gb300 import synth


def test_box_sides_close_the_water_balance_of_one_step():
    terr = synth.make_terrain(40, 60, seed=71, building_frac=0.02)
    p = oracle.Params(ny=40, nx=60)
    hy = synth.hyetograph_constant(90.0, 600.0)
    m = oracle.Member.dry(40, 60)
    oracle.advance(p, terr.z, terr.n, 1.0, 1.0, hy, m, t_end=300.0)
    rate = float(hy[1])
    for (r0, r1, c0, c1) in [(5, 17, 8, 30), (20, 39, 31, 59), (0, 40, 0, 60)]:
        before = m.h[r0:r1, c0:c1].sum() * p.dx * p.dx
        dt, _ = oracle.dt(p, float(m.h.max()), m.t)
        clamp0 = m.clamp
        oracle.step(p, terr.z, terr.n, 1.0, rate, dt, m)
        m.t += dt
        after = m.h[r0:r1, c0:c1].sum() * p.dx * p.dx
        q_in = 0.0
        if c0 > 0:
            q_in += oracle.section_flow(m, p.dx, 0, c0 - 1, r0, r1)    # west side, flowing east
        if r0 > 0:
            q_in += oracle.section_flow(m, p.dx, 1, r0 - 1, c0, c1)    # north side, flowing south
        q_out = oracle.section_flow(m, p.dx, 0, c1 - 1, r0, r1)        # east side
        q_out += oracle.section_flow(m, p.dx, 1, r1 - 1, c0, c1) if r1 < 40 else 0.0
        rain = dt * rate * p.dx * p.dx * (r1 - r0) * (c1 - c0)
        assert m.clamp == clamp0
        assert abs((after - before) - (dt * (q_in - q_out) + rain)) <= 1e-12 * max(before, rain)


def test_uniform_flow_through_a_section_is_the_normal_discharge():
    """A tilted plane with uniform depth h and the Manning normal flux on
    every link (the fixed point of Eq. 2): a section across w cells carries
    w * dx * h^(5/3) S^(1/2) / n."""
    ny, nx, h, S, n = 12, 20, 0.3, 0.004, 0.04
    p = oracle.Params(ny=ny, nx=nx, dt_fixed=0.2, east_outflow=1, edge_slope=S)
    z = np.broadcast_to(S * p.dx * (nx - 1 - np.arange(nx))[None, :], (ny, nx)).copy()
    qn = h ** (5.0 / 3.0) * np.sqrt(S) / n
    m = oracle.Member.dry(ny, nx, np.full((ny, nx), h))
    m.qx[:, 1:] = qn
    oracle.step(p, z, np.full((ny, nx), n), 1.0, 0.0, 0.2, m)
    for c in (3, 10, nx - 1):
        assert np.isclose(oracle.section_flow(m, p.dx, 0, c, 0, ny), ny * p.dx * qn, rtol=1e-12)
    assert oracle.section_flow(m, p.dx, 1, 5, 0, nx) == 0.0
