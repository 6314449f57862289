"""GPU adjoint (flood_adjoint, extension beyond the paper) against the FP64
oracle adjoint and against central finite differences, plus the
torch.autograd.Function wrapper and checkpoint-interval invariance."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import oracle_params, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _wet_case(ny=40, nx=56, M=2, seed=31, depth=0.15):
    terr = synth.make_terrain(ny, nx, seed=seed, building_frac=0.0)
    zmax = float(terr.z.max())
    h0 = np.maximum(depth + 0.4 * (zmax - terr.z) / max(zmax, 1e-6), depth).astype(np.float32)
    rng = np.random.default_rng(seed)
    rm = rng.uniform(0.8, 1.3, M).astype(np.float32)
    sc = rng.uniform(0.8, 1.2, M).astype(np.float32)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    cells = rng.choice(ny * nx, 5, replace=False).astype(np.int32)
    ns, sdt = 8, 30.0
    d = (h0.ravel()[cells][None, :] + rng.normal(0, 0.02, (ns, 5))).astype(np.float64)
    return terr, h0, rm, sc, hy, cells, d, ns, sdt


def _gpu_adjoint(capi, terr, h0, rm, sc, hy, cells, d, sdt, params=None, ckpt=0):
    with capi.Grid(terr.z, terr.n, params) as g:
        g.ensemble_init(len(rm), rm, sc, hy, h0=h0)
        return g.adjoint(cells, d, sdt, ckpt_every=ckpt)


def test_adjoint_matches_fp64_oracle_adjoint(capi):
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case()
    p = capi.Params.default()
    out = _gpu_adjoint(capi, terr, h0, rm, sc, hy, cells, d, sdt, p)
    op = oracle_params(p, *terr.z.shape)
    gn_sum = np.zeros(terr.z.shape)
    for m in range(len(rm)):
        r = oracle.loss_and_grad(op, terr.z, terr.n, float(sc[m]), float(rm[m]), hy, h0, sdt, d,
                                 cells)
        assert abs(out["loss"][m] - r["loss"]) <= 1e-4 * r["loss"]
        assert abs(out["grad_rain"][m] - r["grad_rain"]) <= 2e-3 * abs(r["grad_rain"])
        assert abs(out["grad_scale"][m] - r["grad_scale"]) <= 2e-3 * abs(r["grad_scale"])
        gh = out["grad_h0"][m]
        assert np.max(np.abs(gh - r["grad_h0"])) <= 2e-3 * np.max(np.abs(r["grad_h0"]))
        gn_sum += r["grad_n"]
    assert np.max(np.abs(out["grad_n"] - gn_sum)) <= 2e-3 * np.max(np.abs(gn_sum))


def test_adjoint_agrees_with_central_differences(capi):
    """Fully wet, fixed steps (the schedule the adjoint freezes).  Central
    differences (eps = 1e-3 relative) of the FP64 forward model give the
    reference: the GPU adjoint's rain-multiplier and Manning-scale gradients
    within 1e-3, the per-cell Manning gradient on 32 random wet cells within
    1e-3 (median) and 1e-2 (worst).  Central differences of the GPU's own FP32
    forward (eps = 2e-2, since FP32 rounding of the two runs swamps smaller
    steps, so the difference also carries O(eps^2) curvature) agree within
    5e-2."""
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case(M=1, seed=33)
    hy = synth.hyetograph_constant(100.0, 600.0)
    p = capi.Params.default(dt_fixed=0.5)
    out = _gpu_adjoint(capi, terr, h0, rm, sc, hy, cells, d, sdt, p)
    op = oracle_params(p, *terr.z.shape)
    n64 = terr.n.astype(np.float64)

    def loss64(rm_, sc_, n_=n64):
        return oracle.loss_and_grad(op, terr.z, n_, sc_, rm_, hy, h0, sdt, d, cells)["loss"]

    def loss32(rm_, sc_):
        return _gpu_adjoint(capi, terr, h0, np.array([rm_], np.float32),
                            np.array([sc_], np.float32), hy, cells, d, sdt, p)["loss"][0]

    r0, s0 = float(rm[0]), float(sc[0])
    for key, f64, f32, x0 in (("grad_rain", lambda e: (loss64(r0 + e, s0), loss64(r0 - e, s0)),
                               lambda e: (loss32(r0 + e, s0), loss32(r0 - e, s0)), r0),
                              ("grad_scale", lambda e: (loss64(r0, s0 + e), loss64(r0, s0 - e)),
                               lambda e: (loss32(r0, s0 + e), loss32(r0, s0 - e)), s0)):
        e = 1e-3 * x0
        a, b = f64(e)
        fd = (a - b) / (2 * e)
        assert abs(fd - out[key][0]) <= 1e-3 * abs(fd), (key, fd, out[key][0])
        e32 = 2e-2 * x0  # FP32 rounding of the two runs swamps smaller steps
        a, b = f32(e32)
        fd32 = (a - b) / (2 * e32)
        assert abs(fd32 - out[key][0]) <= 5e-2 * abs(fd), (key, fd32, out[key][0])

    g = out["grad_n"].astype(np.float64)
    rng = np.random.default_rng(7)
    cand = np.nonzero((np.abs(g).ravel() > 1e-2 * np.abs(g).max()) & (h0.ravel() > 0.05))[0]
    pick = rng.choice(cand, 32, replace=False)
    errs = []
    for i in pick:
        e = 1e-3 * n64.flat[i]
        a = n64.copy(); a.flat[i] += e
        b = n64.copy(); b.flat[i] -= e
        fd = (loss64(r0, s0, a) - loss64(r0, s0, b)) / (2 * e)
        errs.append(abs(fd - g.flat[i]) / abs(fd))
    assert np.median(errs) <= 1e-3 and max(errs) <= 1e-2, (np.median(errs), max(errs))


def test_checkpoint_interval_does_not_change_gradients(capi):
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case(M=3, seed=35)
    res = [_gpu_adjoint(capi, terr, h0, rm, sc, hy, cells, d, sdt, ckpt=k) for k in (1, 7, 64, 0)]
    for r in res[1:]:
        for key in ("loss", "grad_rain", "grad_scale"):
            assert np.array_equal(r[key], res[0][key])
        assert np.array_equal(r["grad_n"], res[0]["grad_n"])
        assert np.array_equal(r["grad_h0"], res[0]["grad_h0"])


def test_members_with_different_step_counts(capi):
    """Deep water makes Eq. 4 bind, so members take different numbers of
    steps; each member's gradients still follow the oracle."""
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case(M=3, seed=37, depth=1.2)
    rm = np.array([0.5, 1.0, 3.0], np.float32)
    p = capi.Params.default()
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(3, rm, sc, hy, h0=h0)
        out = g.adjoint(cells, d, sdt)
        steps = g.members()["steps"]
    op = oracle_params(p, *terr.z.shape)
    for m in range(3):
        r = oracle.loss_and_grad(op, terr.z, terr.n, float(sc[m]), float(rm[m]), hy, h0, sdt, d,
                                 cells)
        assert abs(out["loss"][m] - r["loss"]) <= 1e-4 * r["loss"]
        assert abs(out["grad_rain"][m] - r["grad_rain"]) <= 2e-3 * abs(r["grad_rain"])
        assert np.max(np.abs(out["grad_h0"][m] - r["grad_h0"])) <= 2e-3 * np.max(np.abs(r["grad_h0"]))
    assert len(set(steps.tolist())) > 1


def test_autograd_function_returns_the_adjoint_gradients(capi):
    torch = pytest.importorskip("torch")
    from paper_2302_08341_gb300.autograd import gauge_misfit
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case(M=2, seed=39)
    dev = torch.device("cuda")
    n_t = torch.tensor(terr.n, device=dev, requires_grad=True)
    rm_t = torch.tensor(rm, device=dev, requires_grad=True)
    h0_t = torch.tensor(h0, device=dev, requires_grad=True)
    loss = gauge_misfit(n_t, rm_t, h0_t, torch.tensor(terr.z, device=dev),
                        torch.tensor(sc, device=dev), torch.tensor(hy, device=dev), cells, d, sdt)
    loss.backward()
    ref = _gpu_adjoint(capi, terr, np.broadcast_to(h0, (2,) + h0.shape).copy(), rm, sc, hy, cells,
                       d, sdt)
    assert abs(loss.item() - ref["loss"].sum()) <= 1e-12 * ref["loss"].sum()
    assert np.array_equal(n_t.grad.cpu().numpy(), ref["grad_n"])
    assert np.allclose(rm_t.grad.cpu().numpy(), ref["grad_rain"], rtol=1e-6)
    assert np.allclose(h0_t.grad.cpu().numpy(), ref["grad_h0"].sum(axis=0), rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("M,limiter", [(1, 1), (5, 1), (5, 0)])
def test_adjoint_engines_give_bitwise_identical_gradients(capi, M, limiter):
    """Direct-load and TMA-staged replay and reverse stencils: the same
    gradients, bit for bit, on a ragged grid (two spans, partial strips, both
    outflow edges) with members that take different numbers of steps, with
    the limiter compiled in and out."""
    terr, h0, rm, sc, hy, cells, d, ns, sdt = _wet_case(ny=45, nx=150, M=M, seed=39, depth=0.6)
    p = capi.Params.default(south_outflow=1, limiter=limiter)
    res = []
    for engine in (0, 1):
        with capi.Grid(terr.z, terr.n, p) as g:
            g.ensemble_init(M, rm, sc, hy, h0=h0)
            g.set_engine(engine)
            g.set_launch(16, 4 if M >= 4 else 1)
            res.append(g.adjoint(cells, d, sdt, ckpt_every=5))
    for key in ("loss", "grad_rain", "grad_scale", "grad_n", "grad_h0"):
        assert np.array_equal(res[0][key], res[1][key]), key
    assert np.abs(res[0]["grad_n"]).max() > 0


def test_adjoint_at_the_calibration_window_size_follows_the_fp64_adjoint(capi):
    """The adjoint configuration at the size the FP64 oracle adjoint can
    still carry: a 128 x 128 copy of the synthetic city (same generator:
    slope, hills, roads, buildings), one member from a dry start under the
    triangular storm, the loss over 8 gauges sampled every 60 s for 1800 s,
    a checkpoint every 64 steps.  The observations come from a hidden truth
    member run by the oracle.  Against the oracle's reverse mode: loss 1e-4,
    rain-multiplier and Manning-scale gradients 2e-3 relative, the per-cell
    Manning and initial-depth gradients 2e-3 of their largest magnitude.
    Against central differences (1e-3 relative steps) of the FP64 forward
    model: the rain multiplier 1e-3, and the per-cell Manning gradient on 32
    wet cells with the largest gradients (1e-3 median, 1e-2 worst)."""
    import concurrent.futures as cf
    ny = nx = 128
    terr = synth.make_terrain(ny, nx, seed=3)
    hy = synth.hyetograph_triangular(60.0, 1200.0, 3600.0)
    rm, sc = synth.ensemble_prior(3, 1)
    cells = synth.gauge_cells(terr, 8, seed=3)
    p = capi.Params.default()
    op = oracle_params(p, ny, nx)
    z = terr.z.astype(np.float64); n64 = terr.n.astype(np.float64)
    trm, tsc = synth.ensemble_prior(1003, 1)
    truth = oracle.Member.dry(ny, nx)
    obs = []
    for s in range(1, 31):
        oracle.advance(op, z, n64, float(tsc[0]), float(trm[0]), hy, truth, t_end=60.0 * s)
        obs.append(synth.observe(truth.h.ravel()[cells], seed=3, window=s))
    d = np.array(obs)
    with capi.Grid(terr.z, terr.n, p) as g:
        g.ensemble_init(1, rm, sc, hy)
        out = g.adjoint(cells, d, 60.0, ckpt_every=64)
        h_end = g.get_state(0)[0]
    r0, s0 = float(rm[0]), float(sc[0])
    ref = oracle.loss_and_grad(op, z, n64, s0, r0, hy, np.zeros((ny, nx)), 60.0, d, cells)
    assert ref["steps"] >= 1800
    assert abs(out["loss"][0] - ref["loss"]) <= 1e-4 * ref["loss"]
    for key in ("grad_rain", "grad_scale"):
        assert abs(out[key][0] - ref[key]) <= 2e-3 * abs(ref[key]), (key, out[key][0], ref[key])
    for key, got in (("grad_n", out["grad_n"]), ("grad_h0", out["grad_h0"][0])):
        err = np.max(np.abs(got - ref[key])) / np.max(np.abs(ref[key]))
        assert err <= 2e-3, (key, err)

    def loss64(rm_=r0, n_=n64):
        m = oracle.Member.dry(ny, nx)
        L = 0.0
        for s in range(1, 31):
            oracle.advance(op, z, n_, s0, rm_, hy, m, t_end=60.0 * s)
            e = m.h.ravel()[cells] - d[s - 1]
            L += float(np.dot(e, e))
        return L

    g_n = out["grad_n"].astype(np.float64).ravel()
    wet = np.nonzero((h_end.ravel() > 0.01) & (np.abs(g_n) > 1e-3 * np.abs(g_n).max()))[0]
    pick = wet[np.argsort(-np.abs(g_n[wet]))[:32]]
    assert len(pick) == 32

    def fd_cell(i):
        e = 1e-3 * n64.flat[i]
        a = n64.copy(); a.flat[i] += e
        b = n64.copy(); b.flat[i] -= e
        return (loss64(n_=a) - loss64(n_=b)) / (2 * e)

    with cf.ThreadPoolExecutor(max_workers=8) as ex:   # the oracle releases the GIL
        fds = list(ex.map(fd_cell, pick))
        e = 1e-3 * r0
        fr = ex.map(lambda x: loss64(rm_=x), (r0 + e, r0 - e))
        lp, lm = list(fr)
    fd_rain = (lp - lm) / (2 * e)
    assert abs(fd_rain - out["grad_rain"][0]) <= 1e-3 * abs(fd_rain), (fd_rain, out["grad_rain"][0])
    errs = np.array([abs(f - g_n[i]) / abs(f) for f, i in zip(fds, pick)])
    print(f"adjoint 128x128 x 1800 s: {ref['steps']} steps, grad_n max err "
          f"{np.max(np.abs(out['grad_n'] - ref['grad_n'])) / np.max(np.abs(ref['grad_n'])):.2e}, "
          f"FD rain {abs(fd_rain - out['grad_rain'][0]) / abs(fd_rain):.2e}, "
          f"FD cells median {np.median(errs):.2e} worst {errs.max():.2e}")
    assert np.median(errs) <= 1e-3 and errs.max() <= 1e-2, (np.median(errs), errs.max())
