"""Pins of the oracle's calibration step (coarse roughness factor field, its
gradient by the chain rule through the adjoint, and the clipped Polyak step
in log-parameter space): central differences of the forward oracle through
the factor map, the block map's partition of the grid, the identity case of
a field as fine as the grid, and the closed form of one Polyak step on a
residual that is linear in the log-parameters.  CPU only."""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import calibration as CAL


def _wet_case(ny, nx, seed=0):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:ny, 0:nx]
    z = 0.004 * 3.0 * (nx - 1 - xx) + 0.05 * np.sin(0.7 * yy) * np.cos(0.5 * xx)
    n0 = 0.03 + 0.02 * rng.random((ny, nx))
    h0 = 0.35 + 0.1 * np.exp(-((yy - ny / 2) ** 2 + (xx - nx / 3) ** 2) / 8.0)
    return z, n0, h0


def pin_factor_gradient(cal, ny, nx, cy, cx):
    """dL/df from the adjoint's per-cell gradient equals central differences
    of the loss with n = n0 * f[block] (fixed steps, fully wet), on grids the
    blocks do not divide evenly."""
    z, n0, h0 = _wet_case(ny, nx)
    p = oracle.Params(ny=ny, nx=nx, dt_cap=0.5, dt_fixed=0.5)
    hy = np.array([40.0, 10.0]) / 3.6e6
    cells = np.array([2 * nx + 3, 5 * nx + nx // 2, (ny - 2) * nx + nx - 3], np.int32)
    d = np.array([[0.40, 0.33, 0.30], [0.38, 0.35, 0.31]])
    f = 1.0 + 0.2 * np.random.default_rng(3).random((cy, cx))

    def run(fv):
        return oracle.loss_and_grad(p, z, cal.roughness_from_factor(n0, fv), 1.1, 1.3, hy, h0,
                                    20.0, d, cells)

    res = run(f)
    G = cal.factor_grad(n0, res["grad_n"], cy, cx)
    # a small step: a block's perturbation moves many links at once, and a
    # flow reversal (the branch of Eq. 3's max) lies within 1e-6 of f here
    eps = 1e-7
    checked = 0
    for b in range(cy * cx):
        fp = f.copy(); fp.flat[b] += eps
        fm = f.copy(); fm.flat[b] -= eps
        fd = (run(fp)["loss"] - run(fm)["loss"]) / (2 * eps)
        assert abs(fd - G.flat[b]) <= 1e-5 * max(abs(fd), 1e-6 * res["loss"]) + 1e-14
        checked += abs(fd) > 1e-9
    assert checked >= 3  # the loss really depends on several blocks


def pin_block_map(cal):
    """Every fine cell lies in exactly one block; block rows and columns are
    contiguous, non-decreasing and differ in size by at most one."""
    for ny, cy in [(2000, 64), (11, 3), (7, 7), (64, 5)]:
        br, _ = cal.block_index(ny, 1, cy, 1)
        assert br[0] == 0 and br[-1] == cy - 1
        assert np.all(np.diff(br) >= 0) and np.all(np.diff(br) <= 1)
        sizes = np.bincount(br, minlength=cy)
        assert sizes.sum() == ny and sizes.max() - sizes.min() <= 1 and sizes.min() >= 1


def pin_fine_field(cal):
    rng = np.random.default_rng(5)
    n0 = rng.random((6, 9)); gn = rng.standard_normal((6, 9))
    assert np.array_equal(cal.factor_grad(n0, gn, 6, 9), n0 * gn)
    # one block: the plain weighted sum
    assert np.isclose(cal.factor_grad(n0, gn, 1, 1)[0, 0], np.sum(n0 * gn), rtol=1e-14)


def pin_unit_factor(cal):
    rng = np.random.default_rng(6)
    n0 = rng.random((10, 13))
    assert np.array_equal(cal.roughness_from_factor(n0, np.ones((3, 4))), n0)


def pin_polyak_member(cal):
    """For a member whose loss is e(theta)^2 with e linear in theta = log m,
    the step lands where the residual is half the old one (Polyak's step for
    a zero-minimum loss)."""
    a, b, m = 0.3, -0.8, 1.25
    theta = np.log(m)
    e = a + b * theta
    L = e * e
    dL_dm = 2.0 * e * b / m
    m_new, _ = cal.calibration_step([L], [dL_dm], [m], delta=10.0)
    assert np.isclose(a + b * np.log(m_new[0]), e / 2.0, rtol=1e-12)


def pin_polyak_field(cal):
    """Total loss (a + b . log f)^2 over a 2 x 3 field: one step halves the
    residual; with a tight clip every component moves by at most delta."""
    rng = np.random.default_rng(7)
    bvec = rng.standard_normal((2, 3))
    f = 1.0 + 0.1 * rng.random((2, 3))
    a = 0.4
    e = a + np.sum(bvec * np.log(f))
    dL_df = 2.0 * e * bvec / f
    # the total loss is split over two members; their rain steps are zero
    _, f_new = cal.calibration_step([0.7 * e * e, 0.3 * e * e], [0.0, 0.0], [1.0, 1.0], f,
                                    dL_df, delta=10.0)
    assert np.isclose(a + np.sum(bvec * np.log(f_new)), e / 2.0, rtol=1e-12)
    _, f_clip = cal.calibration_step([e * e], [0.0], [1.0], f, dL_df, delta=1e-3)
    assert np.all(np.abs(np.log(f_clip / f)) <= 1e-3 * (1 + 1e-12))


def pin_clip(cal):
    m_new, f_new = cal.calibration_step([4.0, 1.0, 0.0], [1e-9, 0.0, 5.0], [1.0, 2.0, 3.0],
                                        np.ones((1, 2)), np.zeros((1, 2)), delta=0.2)
    assert np.isclose(m_new[0], np.exp(-0.2), rtol=1e-15)   # huge step, clipped
    assert m_new[1] == 2.0                                   # no gradient, no step
    assert m_new[2] == 3.0                                   # zero loss, no step
    assert np.array_equal(f_new, np.ones((1, 2)))            # zero field gradient


def pin_land_first_order(cal):
    """For L_i linear in the log-parameters, the joint step over the rain
    multiplier, the class roughness and the drainage rate changes L_i by
    -eta L_i to first order (no clipping): sum_j G_j step_j = -eta L_i, once,
    not once per parameter group; a member with zero gradient does not move;
    all three groups move together; without class gradients the class
    roughness stays and the rain multiplier and drainage rate still remove
    eta L_i; a tight clip bounds every component."""
    rng = np.random.default_rng(11)
    m = rng.uniform(0.5, 2.0, 3)
    n = rng.uniform(0.02, 0.2, (3, 3))
    d = rng.uniform(1e-6, 5e-6, 3)
    gm = rng.normal(0, 0.5, 3); gm[1] = 0.0
    gc = rng.normal(0, 1.0, (3, 3)); gc[1] = 0.0
    gd = rng.normal(0, 1e5, 3); gd[1] = 0.0
    loss = np.array([0.02, 0.5, 0.03])
    eta = 1e-3

    def change(m2, n2, d2, i, with_class=True):
        dl = m[i] * gm[i] * np.log(m2[i] / m[i]) + d[i] * gd[i] * np.log(d2[i] / d[i])
        if with_class:
            dl += np.sum(n[i] * gc[i] * np.log(n2[i] / n[i]))
        return dl

    m2, n2, d2 = cal.land_step(loss, gm, m, gc, n, gd, d, eta=eta, delta=10.0)
    for i in (0, 2):
        assert np.isclose(change(m2, n2, d2, i), -eta * loss[i], rtol=1e-12)
        assert d2[i] != d[i] and m2[i] != m[i] and np.all(n2[i] != n[i])
    assert m2[1] == m[1] and np.array_equal(n2[1], n[1]) and d2[1] == d[1]
    m4, n4, d4 = cal.land_step(loss, gm, m, None, n, gd, d, eta=eta, delta=10.0)
    assert np.array_equal(n4, n)
    for i in (0, 2):
        assert np.isclose(change(m4, n4, d4, i, with_class=False), -eta * loss[i], rtol=1e-12)
    _, n3, _ = cal.land_step(loss, gm, m, gc, n, gd, d, eta=10.0, delta=0.05)
    assert np.all(np.abs(np.log(n3 / n)) <= 0.05 * (1 + 1e-12))


def pin_land_reduces_to_rain(cal):
    """With zero land-cover gradients the joint step is the rain
    multiplier's own Polyak step (calibration_step without a field)."""
    rng = np.random.default_rng(12)
    m = rng.uniform(0.5, 2.0, 4)
    gm = rng.normal(0, 0.5, 4)
    loss = rng.uniform(0.01, 0.1, 4)
    n = np.full((4, 2), 0.05); d = np.full(4, 2e-6)
    m2, n2, d2 = cal.land_step(loss, gm, m, np.zeros((4, 2)), n, np.zeros(4), d)
    m_ref, _ = cal.calibration_step(loss, gm, m)
    assert np.allclose(m2, m_ref, rtol=1e-15) and np.array_equal(n2, n) and np.array_equal(d2, d)


@pytest.mark.parametrize("ny,nx,cy,cx", [(11, 15, 3, 4), (9, 14, 2, 5)])
def test_factor_gradient_matches_central_differences(ny, nx, cy, cx):
    pin_factor_gradient(CAL, ny, nx, cy, cx)


def test_block_map_partitions_the_grid():
    pin_block_map(CAL)


def test_field_as_fine_as_the_grid_is_the_weighted_cell_gradient():
    pin_fine_field(CAL)


def test_roughness_from_factor_ones_is_the_base_field():
    pin_unit_factor(CAL)


def test_polyak_step_halves_a_linear_residual():
    pin_polyak_member(CAL)


def test_polyak_step_on_the_shared_field():
    pin_polyak_field(CAL)


def test_clip_and_zero_gradient():
    pin_clip(CAL)


def test_land_step_removes_eta_of_a_linear_loss_to_first_order():
    pin_land_first_order(CAL)


def test_land_step_is_the_polyak_step_of_the_calibration_when_only_rain_moves():
    pin_land_reduces_to_rain(CAL)


# plausible mistakes in the calibration oracle; each must fail some pin
MUTATIONS = [
    ("block index rounded up", "return (r * cy) // ny, (c * cx) // nx",
     "return (r * cy + ny - 1) // ny, (c * cx + nx - 1) // nx"),
    ("chain rule without n0", "np.add.at(out, (br[:, None], bc[None, :]), n0 * gn)",
     "np.add.at(out, (br[:, None], bc[None, :]), gn)"),
    ("field gradient not in log space", "G = f * np.asarray(factor_grad_, np.float64)",
     "G = np.asarray(factor_grad_, np.float64)"),
    ("member step without the loss", "step[nz] = _clip(-eta * loss[nz] / gt[nz], delta)",
     "step[nz] = _clip(-eta / gt[nz], delta)"),
    ("member step additive", "m_new = m * np.exp(step)", "m_new = m + step"),
    ("field step takes one member's loss", "L = float(np.sum(loss))", "L = float(loss[0])"),
    ("field step ascends", "np.exp(_clip(-eta * L * G / s2, delta))",
     "np.exp(_clip(eta * L * G / s2, delta))"),
    ("clip one-sided", "return np.minimum(np.maximum(x, -delta), delta)",
     "return np.minimum(x, delta)"),
    ("joint step leaves the rain multiplier out of |G|^2",
     "s2 = Gm * Gm + np.sum(Gn * Gn, axis=1) + Gd * Gd", "s2 = np.sum(Gn * Gn, axis=1) + Gd * Gd"),
    ("joint step leaves the rain multiplier in place",
     "m_new[i] = m[i] * np.exp(_clip(c * Gm[i], delta))", "pass"),
    ("drainage gradient not in log space", "Gd = d * np.asarray(grad_drain, np.float64)",
     "Gd = np.asarray(grad_drain, np.float64)"),
    ("joint step takes the rain multiplier's own Polyak length",
     "c = -eta * loss[i] / s2[i]", "c = -eta * loss[i] / (Gm[i] * Gm[i] + 1e-300)"),
]


def _pins_fail(mod):
    pins = [lambda: pin_factor_gradient(mod, 11, 15, 3, 4), lambda: pin_block_map(mod),
            lambda: pin_fine_field(mod), lambda: pin_unit_factor(mod),
            lambda: pin_polyak_member(mod), lambda: pin_polyak_field(mod), lambda: pin_clip(mod),
            lambda: pin_land_first_order(mod), lambda: pin_land_reduces_to_rain(mod)]
    for pin in pins:
        try:
            pin()
        except Exception:  # a failed pin, or a crash on valid input
            return True
    return False


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_calibration_mistakes(name, old, new):
    with open(os.path.join(os.path.dirname(CAL.__file__), "calibration.py")) as f:
        src = f.read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("calibration_mutant")
    exec(compile(src.replace(old, new), "calibration_mutant.py", "exec"), mod.__dict__)
    assert _pins_fail(mod), name
