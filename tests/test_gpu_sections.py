"""GPU streamflow gauges (discharge through sections of links): equal to the
sums of the members' own links, following the FP64 oracle's trajectory,
consistent with the outflow bookkeeping, and usable as particle-filter
observations with a relative error (Section 4.4)."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _sections(ny, nx):
    return [(0, nx - 1, 0, ny), (0, nx // 2, 3, ny - 5), (1, ny // 3, 2, nx - 7), (1, ny - 1, 0, nx)]


def test_flow_is_the_sum_of_the_members_links(capi):
    ny, nx, M = 45, 150, 4
    terr = synth.make_terrain(ny, nx, seed=81)
    hy = synth.hyetograph_constant(120.0, 600.0)
    rm, sc = synth.ensemble_prior(81, M)
    secs = _sections(ny, nx)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.advance_to(400.0)
        q = g.flow_sample(secs)
        st = [g.get_state(m) for m in range(M)]
    for m in range(M):
        _, qx, qy = st[m]
        for k, (axis, fixed, a, b) in enumerate(secs):
            links = qx[a:b, fixed] if axis == 0 else qy[fixed, a:b]
            want = float(np.sum(links.astype(np.float64))) * 3.0
            assert abs(q[m, k] - want) <= 1e-6 * max(abs(want), 1e-3)
    assert np.all(q[:, 3] == 0.0)          # the south edge is a wall
    assert np.all(q[:, 0] > 0.0)           # water leaves through the east edge


def test_flow_follows_the_oracle_and_the_outflow_bookkeeping(capi):
    ny, nx = 64, 96
    terr = synth.make_terrain(ny, nx, seed=82)
    hy = synth.hyetograph_constant(100.0, 900.0)
    p = capi.Params.default()
    secs = _sections(ny, nx)
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32), hy)
        g.advance_to(600.0)
        q = g.flow_sample(secs)[0]
        out0 = g.volumes()["outflow"][0]
        t0 = g.members()["t"][0]
        g.step(1)
        dt = g.members()["t"][0] - t0
        q1 = g.flow_sample(secs)[0]
        out1 = g.volumes()["outflow"][0]
    # the edge discharge after a step, times the step, is the step's outflow
    assert abs((out1 - out0) - q1[0] * dt) <= 1e-5 * (out1 - out0)
    mo = oracle.Member.dry(ny, nx)
    oracle.advance(oracle_params(p, ny, nx), terr.z, terr.n, 1.0, 1.0, hy, mo, t_end=600.0)
    for k, (axis, fixed, a, b) in enumerate(secs):
        want = oracle.section_flow(mo, p.dx, axis, fixed, a, b)
        assert abs(q[k] - want) <= 1e-3 * max(abs(want), 1e-2), (k, q[k], want)


def test_flows_as_particle_filter_observations(capi):
    """Discharge observations with a relative error sigma = 0.05 d (Section
    4.4) weight the members as the oracle's Eq. 9-12 does."""
    ny, nx, M = 40, 80, 8
    terr = synth.make_terrain(ny, nx, seed=83)
    hy = synth.hyetograph_constant(100.0, 600.0)
    rm, sc = synth.ensemble_prior(83, M)
    secs = [(0, nx - 1, 0, ny), (0, nx // 2, 0, ny)]
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.advance_to(480.0)
        y = g.flow_sample(secs)
        d = y[3].astype(np.float64) * np.array([1.03, 0.97])
        sigma = 0.05 * np.abs(d)
        u, beta = synth.pf_draws(83, 1, M)
        pf = g.pf_assimilate(d, sigma, u, beta, y=y, n_thr_frac=1e-9)
    w_o, neff_o = oracle.pf_weights(y.astype(np.float64), d, sigma, np.full(M, 1.0 / M))
    big = w_o > 1e-300
    assert np.allclose(pf["weights"][big], w_o[big], rtol=1e-6)
    assert abs(pf["neff"] - neff_o) <= 1e-6 * neff_o


def test_sections_outside_the_grid_are_refused(capi):
    terr = synth.make_terrain(20, 30, seed=84)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(1, np.ones(1, np.float32), np.ones(1, np.float32),
                        synth.hyetograph_constant(50.0, 300.0))
        for bad in [(0, 30, 0, 5), (1, 5, 10, 31), (2, 0, 0, 1), (0, 3, 5, 5)]:
            with pytest.raises(capi.FloodError):
                g.flow_sample([bad])
