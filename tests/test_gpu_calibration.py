"""GPU gradient calibration (extension beyond the paper): the coarse roughness
factor field, its gradient from the adjoint against the FP64 oracle adjoint
taken through the oracle's factor map, the calibration step against the
oracle's rule, the order checks, and the full-size ensemble (2000 x 2000
cells, 96 members, 64 x 64 field, one 300 s window) on sampled blocks and
against central differences of the ensemble loss."""
import numpy as np
import pytest

import oracle
from oracle import calibration as cal
from paper_2302_08341_gb300 import synth
from tests.gpu_util import oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _factor(cy, cx, seed):
    return (0.8 + 0.4 * np.random.default_rng(seed).random((cy, cx))).astype(np.float32)


def _fine(n0, f):
    """n0 * f[block] rounded to FP32 once, as the device computes it."""
    br, bc = cal.block_index(n0.shape[0], n0.shape[1], f.shape[0], f.shape[1])
    return (n0.astype(np.float32) * f[np.ix_(br, bc)]).astype(np.float32)


def test_factor_field_is_the_premultiplied_roughness(capi):
    """A run with a factor field equals, bit for bit, a run whose base field
    was multiplied by it beforehand; a second field replaces the first (it
    scales the base field, not the scaled one)."""
    terr = synth.make_terrain(45, 150, seed=41)
    f = _factor(4, 7, 41)
    hy = synth.hyetograph_constant(80.0, 300.0)
    rm, sc = synth.ensemble_prior(41, 3)
    res = []
    for mode in ("factor", "premultiplied"):
        n = terr.n if mode == "factor" else _fine(terr.n, f)
        with capi.Grid(terr.z, n) as g:
            g.ensemble_init(3, rm, sc, hy)
            if mode == "factor":
                g.set_roughness_factor(np.full((2, 3), 1.5, np.float32))
                g.set_roughness_factor(f)
                assert np.array_equal(g.roughness_factor(), f)
            g.advance_to(240.0)
            g.sync()
            res.append([g.get_state(m) for m in range(3)])
    for m in range(3):
        for k in range(3):
            assert np.array_equal(res[0][m][k], res[1][m][k])


def _wet_case(ny, nx, M, seed, ns=4, sdt=30.0):
    terr = synth.make_terrain(ny, nx, seed=seed, building_frac=0.0)
    zmax = float(terr.z.max())
    h0 = np.maximum(0.15 + 0.4 * (zmax - terr.z) / max(zmax, 1e-6), 0.15).astype(np.float32)
    rng = np.random.default_rng(seed)
    rm = rng.uniform(0.8, 1.3, M).astype(np.float32)
    sc = rng.uniform(0.8, 1.2, M).astype(np.float32)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    cells = rng.choice(ny * nx, 5, replace=False).astype(np.int32)
    d = (h0.ravel()[cells][None, :] + rng.normal(0, 0.02, (ns, 5))).astype(np.float64)
    return terr, h0, rm, sc, hy, cells, d, sdt


def test_factor_gradient_and_step_follow_the_oracle(capi):
    ny, nx, M, cy, cx = 40, 56, 3, 3, 4
    terr, h0, rm, sc, hy, cells, d, sdt = _wet_case(ny, nx, M, seed=43)
    f = _factor(cy, cx, 43)
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(M, rm, sc, hy, h0=h0)
        g.set_roughness_factor(f)
        out = g.adjoint(cells, d, sdt, grad_h0=False)
        G = g.roughness_factor_grad()
        loss = g.calibration_step(eta=1.0, delta=0.2)
        mem = g.members()
        f_new = g.roughness_factor()
        with pytest.raises(capi.FloodError):   # the adjoint is spent
            g.calibration_step()
    op = oracle_params(p, ny, nx)
    nf = _fine(terr.n, f)
    gn = np.zeros((ny, nx))
    L_or, gr_or = [], []
    for m in range(M):
        r = oracle.loss_and_grad(op, terr.z, nf, float(sc[m]), float(rm[m]), hy, h0, sdt, d,
                                 cells)
        gn += r["grad_n"]
        L_or.append(r["loss"])
        gr_or.append(r["grad_rain"])
    G_or = cal.factor_grad(terr.n, gn, cy, cx)
    assert np.max(np.abs(G - G_or)) <= 2e-3 * np.max(np.abs(G_or))
    assert np.allclose(loss, out["loss"], rtol=1e-12)
    # the oracle's rule on the GPU's own gradients: the same step to FP32 rounding
    m_or, f_or = cal.calibration_step(out["loss"], out["grad_rain"], rm, f, G)
    assert np.allclose(mem["rain_mult"], m_or, rtol=2e-7)
    assert np.allclose(f_new, f_or, rtol=2e-7)
    assert np.any(np.abs(np.log(f_new / f)) > 1e-3)   # the field really moved
    # and on the oracle's own gradients, within what the adjoint's error allows
    m_or2, f_or2 = cal.calibration_step(L_or, gr_or, rm, f, G_or)
    assert np.allclose(mem["rain_mult"], m_or2, rtol=2e-3)
    assert np.allclose(f_new, f_or2, rtol=2e-3)


def test_rain_only_step_without_a_field(capi):
    terr, h0, rm, sc, hy, cells, d, sdt = _wet_case(32, 40, 4, seed=45)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(4, rm, sc, hy, h0=h0)
        out = g.adjoint(cells, d, sdt, grad_n=False, grad_h0=False)
        g.calibration_step(eta=0.5, delta=0.1)
        mem = g.members()
    m_or, _ = cal.calibration_step(out["loss"], out["grad_rain"], rm, eta=0.5, delta=0.1)
    assert np.allclose(mem["rain_mult"], m_or, rtol=2e-7)


def test_calls_out_of_order_are_refused(capi):
    terr, h0, rm, sc, hy, cells, d, sdt = _wet_case(24, 36, 2, seed=47)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(2, rm, sc, hy, h0=h0)
        with pytest.raises(capi.FloodError):         # no adjoint yet
            g.calibration_step()
        with pytest.raises(capi.FloodError):         # no factor field
            g.roughness_factor_grad()
        for bad in (np.zeros((2, 2), np.float32), np.ones((25, 3), np.float32)):
            with pytest.raises(capi.FloodError):
                g.set_roughness_factor(bad)
        g.set_roughness_factor(np.ones((2, 3), np.float32))
        g.adjoint(cells, d, sdt, grad_n=False, grad_h0=False)
        with pytest.raises(capi.FloodError):         # the field needs grad_n
            g.calibration_step()
        g.adjoint(cells, d, sdt, grad_h0=False)
        g.advance_to(float(g.members()["t"].max()) + 10.0)
        with pytest.raises(capi.FloodError):         # the ensemble moved on
            g.roughness_factor_grad()
        g.adjoint(cells, d, sdt, grad_h0=False)
        with pytest.raises(capi.FloodError):
            g.calibration_step(eta=0.0)
        g.calibration_step()


def test_full_size_ensemble_calibration_window(capi):
    """2000 x 2000 cells, 96 members, a 64 x 64 factor field, one 300 s
    window observed at its end by 6 gauges, in the launch configuration the
    benchmark uses: the block sums of the field gradient on sampled blocks and
    in total against the per-cell gradient, the losses against the gauge
    outputs at the window end, and the step against the oracle's rule."""
    ny = nx = 2000
    M, G, cy, cx = 96, 6, 64, 64
    terr = synth.make_terrain(ny, nx, seed=4)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(4, M)
    cells = synth.gauge_cells(terr, G, seed=4)
    trm, tsc = synth.ensemble_prior(1004, 1)
    with capi.Grid(terr.z, terr.n) as t:
        t.ensemble_init(1, trm, tsc, hy)
        t.advance_to(300.0)
        d = synth.observe(t.gauge_sample(cells)[0], seed=4, window=1)[None, :]
    f = np.ones((cy, cx), np.float32)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.set_roughness_factor(f)
        out = g.adjoint(cells, d, 300.0, grad_h0=False)
        assert np.all(g.members()["t"] == 300.0)
        Gf = g.roughness_factor_grad()
        y = g.gauge_sample(cells)
        loss = g.calibration_step()
        mem = g.members()
        f_new = g.roughness_factor()
    L = np.sum((y.astype(np.float64) - d) ** 2, axis=1)
    assert np.allclose(out["loss"], L, rtol=1e-12) and np.allclose(loss, L, rtol=1e-12)
    w = terr.n.astype(np.float64) * out["grad_n"].astype(np.float64)
    assert abs(Gf.sum() - w.sum()) <= 1e-10 * np.abs(w).sum()
    br, bc = cal.block_index(ny, nx, cy, cx)
    rng = np.random.default_rng(4)
    for b in rng.choice(cy * cx, 8, replace=False):
        rows, cols = br == b // cx, bc == b % cx
        blk = w[np.ix_(rows, cols)]
        assert abs(Gf.flat[b] - blk.sum()) <= 1e-10 * max(np.abs(blk).sum(), 1e-300)
    m_or, f_or = cal.calibration_step(out["loss"], out["grad_rain"], rm, f, Gf)
    assert np.allclose(mem["rain_mult"], m_or, rtol=2e-7)
    assert np.allclose(f_new, f_or, rtol=2e-7)
    assert np.all(np.abs(np.log(f_new)) <= 0.2 * (1 + 1e-6))


def test_full_size_adjoint_against_central_differences(capi):
    """2000 x 2000 cells, 96 members, a 64 x 64 factor field, one 300 s
    window from the dry start observed every 60 s by 6 gauges, in the
    launch configuration the benchmark uses: the adjoint's rain-multiplier,
    Manning-scale and factor-field gradients against central differences of
    the whole ensemble's loss (every member's rain multiplier, every
    member's scale, every factor moved by +-1 %), within 3 % (the
    differences also move the CFL step schedule the adjoint holds fixed)."""
    ny = nx = 2000
    M, G, cy, cx = 96, 6, 64, 64
    terr = synth.make_terrain(ny, nx, seed=4)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(4, M)
    cells = synth.gauge_cells(terr, G, seed=4)
    obs = np.full((5, G), 0.05)
    f = np.ones((cy, cx), np.float32)

    def run(rain_f=1.0, scale_f=1.0, fac_f=1.0, adjoint=False):
        with capi.Grid(terr.z, terr.n) as g:
            g.ensemble_init(M, (rm * np.float32(rain_f)).astype(np.float32),
                            (sc * np.float32(scale_f)).astype(np.float32), hy)
            g.set_roughness_factor((f * np.float32(fac_f)).astype(np.float32))
            if adjoint:
                out = g.adjoint(cells, obs, 60.0, grad_h0=False)
                return out, g.roughness_factor_grad()
            L = np.zeros(M)
            for s in range(1, 6):
                g.advance_to(60.0 * s)
                y = g.gauge_sample(cells).astype(np.float64)
                L += ((y - obs[s - 1]) ** 2).sum(axis=1)
            return L

    out, Gf = run(adjoint=True)
    assert np.allclose(out["loss"], run(), rtol=1e-6)
    eps = 0.01
    for key, kw, want in (
            ("rain", "rain_f", (out["grad_rain"] * rm.astype(np.float64)).sum()),
            ("scale", "scale_f", (out["grad_scale"] * sc.astype(np.float64)).sum()),
            ("factor", "fac_f", (Gf.astype(np.float64) * f).sum())):
        dL = (run(**{kw: 1 + eps}) - run(**{kw: 1 - eps})).sum() / (2 * eps)
        assert want != 0.0 and abs(dL - want) <= 0.03 * abs(dL), (key, dL, want)


def test_full_size_adjoint_matches_the_fp64_adjoint_on_one_member(capi):
    """The calibration's gradients at their full size against the FP64
    oracle's reverse mode: 2000 x 2000 cells, one member of the calibration
    ensemble from 5 cm of water under the storm, 6 gauges observed at 30 s and
    60 s (the oracle keeps the whole trajectory, about 6 GB for these 60 s).
    Loss 1e-4, rain-multiplier and Manning-scale gradients 2e-3 relative, the
    per-cell Manning gradient 2e-3 of its largest magnitude; the factor-field
    gradient follows from it by the chain rule (pinned on the CPU)."""
    ny = nx = 2000
    terr = synth.make_terrain(ny, nx, seed=4)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(4, 1)
    cells = synth.gauge_cells(terr, 6, seed=4)
    h0 = np.full((ny, nx), 0.05, np.float32)
    d = np.array([[0.06] * 6, [0.07] * 6])
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(1, rm, sc, hy, h0=h0)
        out = g.adjoint(cells, d, 30.0, grad_h0=False)
    ref = oracle.loss_and_grad(oracle_params(p, ny, nx), terr.z, terr.n, float(sc[0]), float(rm[0]),
                               hy, h0, 30.0, d, cells)
    assert abs(out["loss"][0] - ref["loss"]) <= 1e-4 * ref["loss"]
    for key in ("grad_rain", "grad_scale"):
        assert abs(out[key][0] - ref[key]) <= 2e-3 * abs(ref[key]), (key, out[key][0], ref[key])
    err = np.max(np.abs(out["grad_n"] - ref["grad_n"])) / np.max(np.abs(ref["grad_n"]))
    print(f"2000x2000 adjoint, 60 s: grad_n max err {err:.2e}, grad_rain "
          f"{abs(out['grad_rain'][0] - ref['grad_rain']) / abs(ref['grad_rain']):.2e}, "
          f"grad_scale {abs(out['grad_scale'][0] - ref['grad_scale']) / abs(ref['grad_scale']):.2e}")
    assert err <= 2e-3, err
