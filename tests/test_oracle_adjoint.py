"""Pins of the oracle's reverse-mode adjoint (gradients of a gauge-misfit
loss through Eq. 1-5 with the step schedule held fixed): central finite
differences of the forward oracle in the fully wet regime, the dot-product
test <J v, w> = <v, J^T w> per step, and a closed form (uniform rain on a
flat box).  CPU only."""
import numpy as np
import pytest

import oracle


def _wet_case(ny=10, nx=14, seed=0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:ny, 0:nx]
    z = 0.004 * 3.0 * (nx - 1 - xx) + 0.05 * np.sin(0.7 * yy) * np.cos(0.5 * xx)
    n = 0.03 + 0.02 * rng.random((ny, nx))
    h0 = 0.35 + 0.1 * np.exp(-((yy - ny / 2) ** 2 + (xx - nx / 3) ** 2) / 8.0)
    return z, n, h0


def _setup():
    z, n, h0 = _wet_case()
    ny, nx = z.shape
    p = oracle.Params(ny=ny, nx=nx, dt_cap=0.5)
    hy = np.array([40.0, 10.0]) / 3.6e6
    cells = np.array([3 * nx + 4, 6 * nx + 9, 8 * nx + 12], np.int32)
    d = np.array([[0.40, 0.33, 0.30], [0.38, 0.35, 0.31], [0.36, 0.34, 0.33]])
    return p, z, n, h0, hy, cells, d


def _loss(p, z, n, scale, rm, hy, h0, d, cells):
    return oracle.loss_and_grad(p, z, n, scale, rm, hy, h0, 20.0, d, cells)["loss"]


def test_gradients_match_central_differences_fully_wet():
    p, z, n, h0, hy, cells, d = _setup()
    # the step schedule must not move under the perturbations: fixed steps
    p.dt_fixed = 0.5
    res = oracle.loss_and_grad(p, z, n, 1.1, 1.3, hy, h0, 20.0, d, cells)
    assert res["loss"] > 0 and res["steps"] == 120
    eps = 1e-6
    fd = (_loss(p, z, n, 1.1, 1.3 + eps, hy, h0, d, cells) -
          _loss(p, z, n, 1.1, 1.3 - eps, hy, h0, d, cells)) / (2 * eps)
    assert abs(fd - res["grad_rain"]) <= 1e-6 * abs(fd) + 1e-12
    fd = (_loss(p, z, n, 1.1 + eps, 1.3, hy, h0, d, cells) -
          _loss(p, z, n, 1.1 - eps, 1.3, hy, h0, d, cells)) / (2 * eps)
    assert abs(fd - res["grad_scale"]) <= 1e-5 * abs(fd) + 1e-12
    rng = np.random.default_rng(1)
    for _ in range(6):
        i = int(rng.integers(0, z.size))
        for name, arr in (("grad_n", n), ("grad_h0", h0)):
            e = eps * max(1.0, abs(arr.flat[i]))
            ap = arr.copy(); ap.flat[i] += e
            am = arr.copy(); am.flat[i] -= e
            if name == "grad_n":
                fd = (_loss(p, z, ap, 1.1, 1.3, hy, h0, d, cells) -
                      _loss(p, z, am, 1.1, 1.3, hy, h0, d, cells)) / (2 * e)
            else:
                fd = (_loss(p, z, n, 1.1, 1.3, hy, ap, d, cells) -
                      _loss(p, z, n, 1.1, 1.3, hy, am, d, cells)) / (2 * e)
            g = res[name].flat[i]
            assert abs(fd - g) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(res[name]).max()), (name, i, fd, g)


@pytest.mark.parametrize("regime", ["wet", "limited", "drying", "outflow", "land_cover"])
def test_dot_product_identity_per_step(regime):
    """<J v, w> = <v, J^T w> for one step, J by central differences of the
    forward step in every input (h, qx, qy, n), J^T by the adjoint; in the
    wet regime, with links held by the limiter, with cells clamped at zero
    depth (limiter off), with a free-outflow edge, and with land cover
    (runoff coefficients, cells that drainage empties, cells it leaves wet)."""
    p, z, n, h0, hy, cells, d = _setup()
    ny, nx = z.shape
    rng = np.random.default_rng(3)
    dt, rate, rm, sc = 0.4, 3e-5, 1.2, 0.9
    h = h0.copy()
    qx = np.zeros((ny, nx + 1)); qy = np.zeros((ny + 1, nx))
    qx[:, 1:nx] = rng.normal(0, 0.05, (ny, nx - 1))
    qy[1:ny, :] = rng.normal(0, 0.05, (ny - 1, nx))
    if regime == "limited":
        h = 0.02 + 0.01 * rng.random((ny, nx))
        z = z + 0.3 * rng.random((ny, nx))
        dt = 2.0
    elif regime == "drying":
        p.limiter = 0
        h = 0.01 + 0.02 * rng.random((ny, nx))
        n = n * 0.05
        qx[:, 1:nx] = rng.normal(0, 0.4, (ny, nx - 1))
    elif regime == "outflow":
        qx[:, nx] = np.abs(rng.normal(0, 0.05, ny))
    elif regime == "land_cover":
        p.east_outflow = 0
        h = 0.002 + 0.004 * rng.random((ny, nx))
        qx[:, 1:nx] = rng.normal(0, 0.002, (ny, nx - 1))
        qy[1:ny, :] = rng.normal(0, 0.002, (ny - 1, nx))
        u = rng.random((ny, nx))
        p.rc = np.ascontiguousarray(np.where(rng.random((ny, nx)) < 0.5, 0.9, 1.0))
        # a third emptied (drainage 2 cm per step), a third drained in part
        p.drain = np.ascontiguousarray(np.where(u < 1 / 3, 0.02 / dt,
                                                np.where(u < 2 / 3, 0.0005 / dt, 0.0)))
    else:
        p.east_outflow = 0
    m = oracle.Member(h=h, qx=qx, qy=qy)
    v = [rng.normal(size=(ny, nx)), rng.normal(size=(ny, nx + 1)),
         rng.normal(size=(ny + 1, nx)), rng.normal(size=(ny, nx))]
    v[1][:, 0] = 0; v[2][0, :] = 0; v[2][ny, :] = 0
    w = [rng.normal(size=(ny, nx)), rng.normal(size=(ny, nx + 1)), rng.normal(size=(ny + 1, nx))]
    w[1][:, 0] = 0; w[2][0, :] = 0; w[2][ny, :] = 0

    def fwd(e):
        mm = oracle.Member(h=m.h + e * v[0], qx=m.qx + e * v[1], qy=m.qy + e * v[2])
        oracle.step(p, z, n + e * v[3], sc, rate * rm, dt, mm)
        return mm

    base = fwd(0.0)
    if regime == "limited":
        lim = np.where(base.qx[:, 1:nx] > 0, h[:, :-1], h[:, 1:]) * p.dx / (4 * dt)
        assert np.isclose(np.abs(base.qx[:, 1:nx]), lim, rtol=1e-13).sum() >= 3
    if regime == "drying":
        assert (base.h == 0).sum() >= 3
    if regime == "land_cover":
        assert (base.h == 0).sum() >= 10 and (base.h[u > 1 / 3] > 0).all()
    e = 1e-7
    a, b = fwd(e), fwd(-e)
    Jv = [(a.h - b.h) / (2 * e), (a.qx - b.qx) / (2 * e), (a.qy - b.qy) / (2 * e)]
    lhs = sum(float((x * y).sum()) for x, y in zip(Jv, w))
    lh, lqx, lqy = w[0].copy(), w[1].copy(), w[2].copy()
    gn, _, _ = oracle.step_adjoint(p, z, n, sc, rate, rm, dt, m, lh, lqx, lqy)
    rhs = float((v[0] * lh).sum() + (v[1] * lqx).sum() + (v[2] * lqy).sum() + (v[3] * gn).sum())
    assert abs(lhs - rhs) <= 1e-6 * (abs(lhs) + abs(rhs))


def test_closed_form_uniform_rain_on_flat_box():
    """No flow on a flat closed box: h(T) = h0 + m r T at every cell, so
    L = sum_s (h0 + m r t_s - d_s)^2 at one gauge gives
    dL/dm = sum_s 2 (h(t_s) - d_s) r t_s; raising h0 everywhere keeps the
    surface flat, so sum_i dL/dh0_i = sum_s 2 (h(t_s) - d_s); with no flow
    there is no Manning sensitivity."""
    ny, nx = 6, 7
    p = oracle.Params(ny=ny, nx=nx, east_outflow=0, dt_cap=0.7)
    z = np.full((ny, nx), 2.0); n = np.full((ny, nx), 0.04)
    r = 30.0 / 3.6e6
    hy = np.array([r])
    cells = np.array([2 * nx + 3], np.int32)
    d = np.array([[0.01], [0.02], [0.015]])
    h0 = np.full((ny, nx), 0.005)
    res = oracle.loss_and_grad(p, z, n, 1.0, 1.7, hy, h0, 50.0, d, cells)
    t = np.array([50.0, 100.0, 150.0])
    hT = 0.005 + 1.7 * r * t
    assert abs(res["loss"] - ((hT - d[:, 0]) ** 2).sum()) < 1e-15
    assert abs(res["grad_rain"] - (2 * (hT - d[:, 0]) * r * t).sum()) < 1e-12
    assert abs(res["grad_h0"].sum() - (2 * (hT - d[:, 0])).sum()) < 1e-12
    assert not res["grad_n"].any() and res["grad_scale"] == 0.0
