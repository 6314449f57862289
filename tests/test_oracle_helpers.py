"""Pins of the oracle's helpers that the scheme pins do not reach: the maximum
depth that feeds Eq. 4 inside the member's evolution (Eq. 6), the gauge
sample of DA step (I) (Section 3.3), and the ensemble loop that evolves every
member independently (Eq. 6 for each particle).  CPU only.

- The maximum depth is reached through orc_advance, the way the evolution uses
  it: on a closed flat box at rest the depth never changes, so every step must
  take exactly Eq. 4's k dx / sqrt(g h) at Section 4.1's 4.2 m; with one deep
  cell in a shallow field the deep cell (not the mean, not the first row)
  decides the step, and the second step follows numpy's maximum of the state
  the first step left.
- The gauge sample reads member m, cell i of a field filled with
  1000 m + i, so every sample names the member and cell it came from.
- The ensemble loop must give every member exactly what orc_advance gives it
  alone, on one thread and on four."""
import math

import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth


def _flat_box(ny, nx, dt_cap):
    return oracle.Params(ny=ny, nx=nx, dt_cap=dt_cap, rain_block=1e9, east_outflow=0)


def test_steps_at_rest_take_eq4_of_section_4_1_depth():
    """Flat closed box, uniform 4.2 m (Section 4.1's maximum depth), no rain:
    a lake at rest, so each step's length is alpha dx / sqrt(g 4.2)."""
    ny, nx = 6, 9
    p = _flat_box(ny, nx, dt_cap=10.0)
    z = np.zeros((ny, nx)); n = np.full((ny, nx), 0.05)
    m = oracle.Member.dry(ny, nx, np.full((ny, nx), 4.2))
    dts = oracle.advance(p, z, n, 1.0, 1.0, np.zeros(1), m, max_steps=3, log_dt=True)
    want = 0.7 * 3.0 / math.sqrt(9.81 * 4.2)
    assert len(dts) == 3
    for d in dts:
        assert abs(d - want) <= 1e-15 * want
    assert np.all(m.h == 4.2)
    assert abs(m.t - 3 * want) <= 1e-14


@pytest.mark.parametrize("where", [(0, 0), (5, 7), (2, 3), (5, 0)])
def test_the_deepest_cell_decides_the_step(where):
    """0.05 m everywhere except one 2 m cell: the first step is Eq. 4 at 2 m
    wherever the cell lies (a mean, a partial scan or a minimum would give a
    longer step); the second is Eq. 4 at numpy's maximum of the state after
    the first step."""
    ny, nx = 6, 8
    p = _flat_box(ny, nx, dt_cap=10.0)
    z = np.zeros((ny, nx)); n = np.full((ny, nx), 0.05)
    h0 = np.full((ny, nx), 0.05); h0[where] = 2.0
    m = oracle.Member.dry(ny, nx, h0)
    d1 = oracle.advance(p, z, n, 1.0, 1.0, np.zeros(1), m, max_steps=1, log_dt=True)[0]
    assert abs(d1 - 0.7 * 3.0 / math.sqrt(9.81 * 2.0)) <= 1e-15 * d1
    hm = float(np.max(m.h))
    assert 0.05 < hm < 2.0      # the column has started to spread
    assert oracle.hmax(m.h) == hm
    d2 = oracle.advance(p, z, n, 1.0, 1.0, np.zeros(1), m, max_steps=1, log_dt=True)[0]
    assert abs(d2 - 0.7 * 3.0 / math.sqrt(9.81 * hm)) <= 1e-15 * d2


def test_gauge_sample_reads_the_member_and_cell_it_names():
    M, ny, nx = 3, 5, 7
    h = np.empty((M, ny, nx))
    for mm in range(M):
        h[mm] = 1000.0 * mm + np.arange(ny * nx).reshape(ny, nx)
    cells = np.array([0, 8, 34, 17, 20], np.int32)
    y = oracle.gauge_sample(h, cells)
    assert y.shape == (M, len(cells))
    for mm in range(M):
        for g, c in enumerate(cells):
            assert y[mm, g] == 1000.0 * mm + c


@pytest.mark.parametrize("nthreads", [1, 4])
def test_ensemble_loop_equals_each_member_alone(nthreads):
    """Members of different Manning scale and rain multiplier, rain on an
    urban DEM with free outflow, 150 s: the ensemble loop's state, clock,
    step count and volumes are bit for bit those of orc_advance per member."""
    ny, nx, M = 20, 28, 4
    terr = synth.make_terrain(ny, nx, seed=7)
    hy = synth.hyetograph_constant(200.0, 600.0)
    rm = np.array([0.7, 1.0, 1.3, 2.0]); sc = np.array([1.2, 0.8, 1.0, 0.6])
    p = oracle.Params(ny=ny, nx=nx)
    t0 = [0.0, 0.0, 30.0, 0.0]               # one member starts later
    ens = oracle.Ensemble(p, M)
    ens.t[:] = t0
    steps = ens.advance(terr.z, terr.n, sc, rm, hy, t_end=150.0, nthreads=nthreads)
    vols = ens.volumes()
    for mm in range(M):
        one = oracle.Member.dry(ny, nx)
        one.t = t0[mm]
        k = oracle.advance(p, terr.z, terr.n, float(sc[mm]), float(rm[mm]), hy, one, t_end=150.0)
        assert steps[mm] == k
        assert ens.t[mm] == one.t == 150.0
        assert np.array_equal(ens.h[mm], one.h)
        assert np.array_equal(ens.qx[mm], one.qx)
        assert np.array_equal(ens.qy[mm], one.qy)
        assert np.array_equal(vols[mm], [one.rain, one.outflow, one.clamp, one.drained,
                                         one.inflow])
    assert vols[:, 0].min() > 0 and len(set(steps.tolist())) > 1
