"""GPU reverse mode across land cover (Section 4.1, Table 1): each member's
class roughness as its n field, the rain gradient weighed by the runoff
coefficient, drainage that empties a cell passing no sensitivity, the
drainage rate's gradient; against the FP64 oracle's adjoint with the same
land cover, per-class Manning gradients, closed forms, and bit for bit
across engines."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import oracle_params, require_gpu
from tests.test_gpu_land_cover import _oracle_fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _wet_land_case(ny=40, nx=64, M=2, seed=71):
    """Wet everywhere inside the domain (so every derivative is taken away
    from the wet/dry kinks), the classes of the synthetic city with two
    outside corners, drainage on hardened ground below the water present."""
    terr = synth.make_terrain(ny, nx, seed=seed, building_frac=0.0)
    cls = synth.land_cover(terr, seed=seed, n_ponds=3, pond_side=(4, 9))
    outside = cls == 3
    zmax = float(terr.z.max())
    h0 = np.maximum(0.15 + 0.4 * (zmax - terr.z) / max(zmax, 1e-6), 0.15).astype(np.float32)
    h0[outside] = 0.0
    rng = np.random.default_rng(seed)
    rm = rng.uniform(0.8, 1.3, M).astype(np.float32)
    sc = rng.uniform(0.8, 1.2, M).astype(np.float32)
    n_m, d_m = synth.land_prior(seed, M)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    inside = np.flatnonzero(~outside.ravel())
    cells = inside[np.linspace(0, inside.size - 1, 5).astype(int)].astype(np.int32)
    ns, sdt = 5, 30.0
    d = (h0.ravel()[cells][None, :] + rng.normal(0, 0.02, (ns, cells.size))).astype(np.float64)
    return terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt


def _gpu_adjoint(capi, case, engine=None, shape=None, ckpt_every=0):
    terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt = case
    with capi.Grid(terr.z, terr.n, capi.Params.default()) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(len(rm), rm, sc, hy, h0=h0)
        g.set_land_params(n_m, d_m)
        if engine is not None:
            g.set_engine(engine)
        if shape is not None:
            g.set_launch(*shape)
        out = g.adjoint(cells, d, sdt, ckpt_every=ckpt_every)
        out["class"], out["drain"] = g.adjoint_land_grad()
    return out


def test_land_cover_adjoint_matches_the_oracle_adjoint(capi):
    case = _wet_land_case()
    terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt = case
    ny, nx = terr.z.shape
    out = _gpu_adjoint(capi, case)
    p = capi.Params.default()
    gn_sum = np.zeros((ny, nx))
    for m in range(len(rm)):
        z, n, rc, dr, _ = _oracle_fields(terr, cls, n_m[m], d_m[m])
        op = oracle_params(p, ny, nx)
        op.rc, op.drain = rc, dr
        r = oracle.loss_and_grad(op, z, n, float(sc[m]), float(rm[m]), hy, h0.astype(np.float64),
                                 sdt, d, cells)
        assert abs(out["loss"][m] - r["loss"]) <= 1e-4 * r["loss"]
        assert abs(out["grad_rain"][m] - r["grad_rain"]) <= 2e-3 * abs(r["grad_rain"])
        assert abs(out["grad_scale"][m] - r["grad_scale"]) <= 2e-3 * abs(r["grad_scale"])
        gh = out["grad_h0"][m]
        assert np.max(np.abs(gh - r["grad_h0"])) <= 2e-3 * np.max(np.abs(r["grad_h0"]))
        gn_sum += r["grad_n"]
        # the oracle differentiates a factor on the drainage field; the
        # device, the member's drainage rate (the field's value where it drains)
        want_d = r["grad_drain"] / float(d_m[m])
        assert want_d != 0.0
        assert abs(out["drain"][m] - want_d) <= 2e-3 * abs(want_d)
        want = np.array([r["grad_n"][cls == k].sum() for k in range(4)])
        got = out["class"][m]
        assert np.all(np.abs(got - want) <= 2e-3 * np.max(np.abs(want)) + 1e-12), (m, got, want)
    assert np.max(np.abs(out["grad_n"] - gn_sum)) <= 2e-3 * np.max(np.abs(gn_sum))
    # the runoff weighting matters here: green land keeps 90 % of the rain
    assert np.any(cls == 0) and np.any(cls == 2)


def test_drainage_that_empties_every_cell_passes_nothing(capi):
    """Closed form: a flat closed box of hardened ground whose drainage per
    step exceeds the rain that falls on it stays dry; the gauge depths (0)
    depend neither on the initial depths nor on the rain multiplier."""
    ny, nx = 12, 40
    z = np.zeros((ny, nx), np.float32)
    n = np.full((ny, nx), 0.03, np.float32)
    cls = np.full((ny, nx), 2, np.uint8)
    p = capi.Params.default(east_outflow=0)
    hy = synth.hyetograph_constant(30.0, 600.0)
    cells = np.array([5 * nx + 7, 9 * nx + 30], np.int32)
    d = np.array([[0.01, 0.02], [0.015, 0.01]])
    for engine in (0, 1):
        with capi.Grid(z, n, p) as g:
            g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(2, np.ones(2, np.float32), np.ones(2, np.float32), hy)
            g.set_land_params(drain_rate=np.full(2, 100.0 / 3.6e6, np.float32))
            g.set_engine(engine)
            out = g.adjoint(cells, d, 60.0)
            cg, gd = g.adjoint_land_grad()
        assert np.allclose(out["loss"], (d ** 2).sum(), rtol=1e-12)
        assert np.all(out["grad_h0"] == 0.0) and np.all(out["grad_rain"] == 0.0)
        assert np.all(out["grad_n"] == 0.0) and np.all(cg == 0.0) and np.all(gd == 0.0)


def test_drainage_gradient_closed_form(capi):
    """Closed form: on a flat closed box of hardened ground whose rain r m
    exceeds its drainage d, h(t) = (r m - d) t everywhere; with
    e = h(t_s) - obs_s, dL/dd = -sum 2 e t_s and dL/dm = sum 2 e r t_s."""
    ny, nx = 12, 40
    z = np.zeros((ny, nx), np.float32)
    n = np.full((ny, nx), 0.03, np.float32)
    cls = np.full((ny, nx), 2, np.uint8)
    p = capi.Params.default(east_outflow=0)
    r, dr = 60.0 / 3.6e6, 12.0 / 3.6e6
    hy = synth.hyetograph_constant(60.0, 600.0)
    rm = np.array([1.0, 1.3], np.float32)
    cells = np.array([5 * nx + 7, 9 * nx + 30], np.int32)
    ts = 30.0 * np.arange(1, 5)
    obs = np.array([[0.0004, 0.0009]] * 4) * np.arange(1, 5)[:, None]
    for engine in (0, 1):
        with capi.Grid(z, n, p) as g:
            g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(2, rm, np.ones(2, np.float32), hy)
            g.set_land_params(drain_rate=np.full(2, dr, np.float32))
            g.set_engine(engine)
            out = g.adjoint(cells, obs, 30.0)
            _, gd = g.adjoint_land_grad(classes=False)
        for m in range(2):
            rate = float(np.float32(hy[0])) * float(rm[m])
            e = (rate - float(np.float32(dr))) * ts[:, None] - obs
            assert abs(out["loss"][m] - (e ** 2).sum()) <= 1e-4 * (e ** 2).sum()
            want_d = -(2 * e * ts[:, None]).sum()
            assert abs(gd[m] - want_d) <= 1e-3 * abs(want_d)
            want_r = (2 * e * float(np.float32(hy[0])) * ts[:, None]).sum()
            assert abs(out["grad_rain"][m] - want_r) <= 1e-3 * abs(want_r)


@pytest.mark.parametrize("M,shape", [(1, (16, 1)), (5, (16, 4)), (5, (32, 4))])
def test_land_cover_adjoint_engines_bitwise(capi, M, shape):
    """Direct-load and TMA-staged logged forward, replay and reverse stencil
    with land cover: the same loss and gradients, bit for bit."""
    case = _wet_land_case(ny=45, nx=150, M=M, seed=72)
    res = [_gpu_adjoint(capi, case, engine=e, shape=shape, ckpt_every=5) for e in (0, 1)]
    for key in ("loss", "grad_rain", "grad_scale", "grad_n", "grad_h0", "class", "drain"):
        assert np.array_equal(res[0][key], res[1][key]), key


def test_land_cover_adjoint_refusals(capi):
    terr = synth.make_terrain(24, 30, seed=73)
    cls = synth.land_cover(terr, seed=73, pond_side=(3, 5))
    hy = synth.hyetograph_constant(50.0, 300.0)
    with capi.Grid(terr.z, terr.n) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(2, np.ones(2, np.float32), np.ones(2, np.float32), hy)
        with pytest.raises(capi.FloodError):   # no adjoint yet
            g.adjoint_land_grad()
        with pytest.raises(capi.FloodError):   # the roughness comes from the classes
            g.set_roughness_factor(np.ones((2, 2), np.float32))
        g.adjoint(np.array([40], np.int32), np.zeros((1, 1)), 30.0, grad_n=False)
        with pytest.raises(capi.FloodError):   # that adjoint had no Manning gradient
            g.adjoint_land_grad()
        _, gd = g.adjoint_land_grad(classes=False)  # the drainage gradient needs none
        assert gd.shape == (2,)
    with capi.Grid(terr.z, terr.n) as g:
        g.set_roughness_factor(np.ones((2, 2), np.float32))
        with pytest.raises(capi.FloodError):   # land cover would replace the factor field
            g.set_land_cover(cls, synth.LAND_CLASSES)


def test_autograd_function_with_land_cover(capi):
    """The torch.autograd.Function over the land-cover adjoint returns the
    C ABI's gradients for the class roughness, drainage rate, rain
    multiplier and initial depth."""
    torch = pytest.importorskip("torch")
    from paper_2302_08341_gb300.autograd import land_gauge_misfit
    case = _wet_land_case(M=2, seed=74)
    terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt = case
    ref = _gpu_adjoint(capi, case)
    dev = torch.device("cuda")
    nc_t = torch.tensor(n_m, device=dev, requires_grad=True)
    dr_t = torch.tensor(d_m, device=dev, requires_grad=True)
    rm_t = torch.tensor(rm, device=dev, requires_grad=True)
    h0_t = torch.tensor(h0, device=dev, requires_grad=True)
    loss = land_gauge_misfit(nc_t, dr_t, rm_t, h0_t, torch.tensor(terr.z, device=dev),
                             torch.tensor(terr.n, device=dev), cls, synth.LAND_CLASSES,
                             torch.tensor(sc, device=dev), torch.tensor(hy, device=dev), cells, d,
                             sdt)
    loss.backward()
    assert abs(loss.item() - ref["loss"].sum()) <= 1e-12 * ref["loss"].sum()
    assert np.allclose(nc_t.grad.cpu().numpy(), ref["class"], rtol=1e-6)
    assert np.allclose(dr_t.grad.cpu().numpy(), ref["drain"], rtol=1e-6)
    assert np.allclose(rm_t.grad.cpu().numpy(), ref["grad_rain"], rtol=1e-6)
    assert np.allclose(h0_t.grad.cpu().numpy(), ref["grad_h0"].sum(axis=0), rtol=1e-5, atol=1e-9)


def test_full_size_land_cover_adjoint_window(capi):
    """2000 x 2000 cells, 96 members with their own class roughness and
    drainage rate, as the benchmark runs them: one 300 s window's adjoint
    after a 300 s spin-up against central differences of the whole
    ensemble's loss in the drainage rates (+-5 %) and the rain multipliers
    (+-1 %) over that window (the differences also move the CFL step
    schedule, which the adjoint holds fixed: a small effect here, inside the
    3 % allowed), and the per-class gradients against the Manning gradient
    field."""
    ny = nx = 2000
    M = 96
    terr = synth.make_terrain(ny, nx, seed=1)
    cls = synth.land_cover(terr, seed=1)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(1, M)
    n_m, d_m = synth.land_prior(1, M)
    p = capi.Params.default()
    cells = synth.gauge_cells(terr, 6, seed=1)
    cells = cells[cls.ravel()[cells] != 3]
    obs = np.full((5, len(cells)), 0.1)

    def run(drain_f=1.0, rain_f=1.0, adjoint=False):
        with capi.Grid(terr.z, terr.n, p) as g:
            g.set_land_cover(cls, synth.LAND_CLASSES)
            g.ensemble_init(M, rm, sc, hy)
            g.set_land_params(n_m, d_m)
            g.advance_to(300.0)
            # the adjoint takes the state at 300 s as its input: the inputs
            # are perturbed for the window alone
            g.set_members(rain_mult=(rm * np.float32(rain_f)).astype(np.float32))
            g.set_land_params(drain_rate=(d_m * np.float32(drain_f)).astype(np.float32))
            if adjoint:
                out = g.adjoint(cells, obs, 60.0)
                gc, gd = g.adjoint_land_grad()
                return out, gc, gd
            L = np.zeros(M)
            for s in range(1, 6):
                g.advance_to(300.0 + 60.0 * s)
                y = g.gauge_sample(cells).astype(np.float64)
                L += ((y - obs[s - 1]) ** 2).sum(axis=1)
            return L

    out, gc, gd = run(adjoint=True)
    L0 = run()
    assert np.allclose(out["loss"], L0, rtol=1e-6)
    eps = 0.05
    dL = (run(drain_f=1 + eps) - run(drain_f=1 - eps)).sum()
    want = (gd * d_m.astype(np.float64)).sum() * 2 * eps
    assert abs(want) > 0 and abs(dL - want) <= 0.03 * abs(dL), (dL, want)
    eps = 0.01
    dL = (run(rain_f=1 + eps) - run(rain_f=1 - eps)).sum()
    want = (out["grad_rain"] * rm.astype(np.float64)).sum() * 2 * eps
    assert abs(dL - want) <= 0.03 * abs(dL), (dL, want)
    # the class gradients partition the member-summed Manning gradient field
    tot = float(out["grad_n"].astype(np.float64).sum())
    assert abs(gc.sum() - tot) <= 1e-3 * np.abs(out["grad_n"]).astype(np.float64).sum()


def test_calibration_step_moves_the_land_parameters_by_the_oracle_rule(capi):
    """With land cover the calibration step takes one joint step per member
    over its rain multiplier, class roughness and drainage rate, by the
    oracle's rule applied to the adjoint's gradients (so the member's loss
    moves by -eta L_i to first order once, not once per parameter group)."""
    from oracle import calibration as cal
    case = _wet_land_case(M=3, seed=75)
    terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt = case
    with capi.Grid(terr.z, terr.n, capi.Params.default()) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(len(rm), rm, sc, hy, h0=h0)
        g.set_land_params(n_m, d_m)
        out = g.adjoint(cells, d, sdt, grad_h0=False)
        gc, gd = g.adjoint_land_grad()
        n0, d0 = g.land_params()
        rm0 = g.members()["rain_mult"]
        loss = g.calibration_step()
        n1, d1 = g.land_params()
        rm1 = g.members()["rain_mult"]
        with pytest.raises(capi.FloodError):   # the gradients are spent
            g.calibration_step()
    assert np.allclose(loss, out["loss"], rtol=1e-12)
    m_or, n_or, d_or = cal.land_step(out["loss"], out["grad_rain"], rm0, gc, n0, gd, d0)
    assert np.allclose(n1, n_or, rtol=2e-7) and np.allclose(d1, d_or, rtol=2e-7)
    assert np.allclose(rm1, m_or, rtol=2e-7)
    assert not np.allclose(n1, n0, rtol=1e-6) and np.all(d1 != d0) and np.all(rm1 != rm0)
    # the separate rain step it replaces moves the multipliers at least as far
    # (further where neither step is clipped)
    m_sep, _ = cal.calibration_step(out["loss"], out["grad_rain"], rm0)
    step_joint = np.abs(np.log(rm1.astype(np.float64) / rm0))
    step_sep = np.abs(np.log(m_sep / rm0))
    assert np.all(step_joint <= step_sep + 1e-6) and np.any(step_joint < step_sep - 1e-3)


def test_calibration_step_without_manning_gradients_moves_rain_and_drainage(capi):
    """An adjoint without grad_n still allows the step: the class roughness
    stays and the joint step runs over the rain multiplier and the drainage
    rate, by the oracle's rule without class gradients."""
    from oracle import calibration as cal
    case = _wet_land_case(M=3, seed=76)
    terr, cls, h0, rm, sc, n_m, d_m, hy, cells, d, sdt = case
    with capi.Grid(terr.z, terr.n, capi.Params.default()) as g:
        g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(len(rm), rm, sc, hy, h0=h0)
        g.set_land_params(n_m, d_m)
        out = g.adjoint(cells, d, sdt, grad_h0=False, grad_n=False)
        _, gd = g.adjoint_land_grad(classes=False)
        n0, d0 = g.land_params()
        rm0 = g.members()["rain_mult"]
        loss = g.calibration_step()
        n1, d1 = g.land_params()
        rm1 = g.members()["rain_mult"]
    assert np.allclose(loss, out["loss"], rtol=1e-12)
    m_or, n_or, d_or = cal.land_step(out["loss"], out["grad_rain"], rm0, None, n0, gd, d0)
    assert np.array_equal(n1, n0)
    assert np.allclose(d1, d_or, rtol=2e-7) and np.allclose(rm1, m_or, rtol=2e-7)
    assert np.all(d1 != d0) and np.all(rm1 != rm0)
