"""FP64 oracle of the ensemble gradient calibration step (test infrastructure
only; the library never imports it).

The paper estimates its uncertain inputs with the particle filter alone
(Section 2.2, Section 4.4); calibrating them by gradients before each filter
update is an extension.  Its pieces, written out plainly:

* a coarse multiplicative roughness field f of cy x cx blocks over the base
  Manning field n0: fine cell (r, c) lies in block (floor(r cy / ny),
  floor(c cx / nx)) and uses n = n0 * f[block];
* the chain rule through that map: dL/df_b = sum over the cells of block b of
  n0 * dL/dn, with dL/dn the adjoint's per-cell Manning gradient;
* one descent step in log-parameter space with the Polyak step length of a
  loss whose minimum is zero, step = -eta * L * g / |g|^2 for the gradient g
  with respect to the log-parameters, every component clipped to
  [-delta, delta]: per member for its rain multiplier (its own loss L_i),
  jointly for the shared factor field (the total loss L = sum_i L_i), and,
  with land cover (Section 4.1), one joint step per member over all of its
  parameters -- rain multiplier, Manning n of every class and drainage rate --
  for its own loss L_i (a separate step on the rain multiplier beside one on
  the land-cover parameters would remove 2 eta L_i to first order).
"""
from __future__ import annotations

import numpy as np


def block_index(ny: int, nx: int, cy: int, cx: int):
    """Coarse row of every fine row and coarse column of every fine column."""
    r = np.arange(ny, dtype=np.int64)
    c = np.arange(nx, dtype=np.int64)
    return (r * cy) // ny, (c * cx) // nx


def roughness_from_factor(n0, f):
    """n = n0 * f[block(r, c)] (FP64)."""
    n0 = np.asarray(n0, np.float64)
    f = np.asarray(f, np.float64)
    br, bc = block_index(n0.shape[0], n0.shape[1], f.shape[0], f.shape[1])
    return n0 * f[np.ix_(br, bc)]


def factor_grad(n0, grad_n, cy: int, cx: int):
    """dL/df for n = n0 * f[block]: the n0-weighted per-cell gradient summed
    over each block."""
    n0 = np.asarray(n0, np.float64)
    gn = np.asarray(grad_n, np.float64)
    br, bc = block_index(n0.shape[0], n0.shape[1], cy, cx)
    out = np.zeros((cy, cx))
    np.add.at(out, (br[:, None], bc[None, :]), n0 * gn)
    return out


def _clip(x, delta):
    return np.minimum(np.maximum(x, -delta), delta)


def calibration_step(loss, grad_rain, rain_mult, factor=None, factor_grad_=None, eta=1.0,
                     delta=0.2):
    """One step on the rain multipliers m_i (per member) and, when given, the
    shared factor field f.  loss[i] = L_i, grad_rain[i] = dL_i/dm_i,
    factor_grad_ = dL/df with L = sum_i L_i.  Returns (new m, new f)."""
    loss = np.asarray(loss, np.float64)
    g = np.asarray(grad_rain, np.float64)
    m = np.asarray(rain_mult, np.float64)
    gt = m * g                                    # dL_i / d(log m_i)
    step = np.zeros_like(m)
    nz = gt != 0.0
    step[nz] = _clip(-eta * loss[nz] / gt[nz], delta)
    m_new = m * np.exp(step)
    if factor is None:
        return m_new, None
    f = np.asarray(factor, np.float64)
    G = f * np.asarray(factor_grad_, np.float64)  # dL / d(log f_b)
    s2 = float(np.sum(G * G))
    L = float(np.sum(loss))
    f_new = f * np.exp(_clip(-eta * L * G / s2, delta)) if s2 > 0.0 else f.copy()
    return m_new, f_new


def land_step(loss, grad_rain, rain_mult, grad_class, n_class, grad_drain, drain, eta=1.0,
              delta=0.2):
    """One joint step per member over theta_i = (m_i, n_i1 .. n_iK, d_i), its
    rain multiplier, class roughness and drainage rate: G = theta_i *
    dL_i/dtheta_i (the log-parameter gradient), step = clip(-eta L_i G /
    |G|^2, delta), no step where |G| = 0.  To first order (no clipping) the
    member's loss changes by sum_j G_j step_j = -eta L_i.  grad_class may be
    None (no per-cell Manning gradients): the class roughness then stays and
    the step runs over (m_i, d_i).  Returns (new m [M], new n_class [M][K],
    new drain [M])."""
    loss = np.asarray(loss, np.float64)
    m = np.asarray(rain_mult, np.float64)
    n = np.asarray(n_class, np.float64)
    d = np.asarray(drain, np.float64)
    Gm = m * np.asarray(grad_rain, np.float64)
    Gn = np.zeros_like(n) if grad_class is None else n * np.asarray(grad_class, np.float64)
    Gd = d * np.asarray(grad_drain, np.float64)
    s2 = Gm * Gm + np.sum(Gn * Gn, axis=1) + Gd * Gd
    m_new, n_new, d_new = m.copy(), n.copy(), d.copy()
    for i in range(len(loss)):
        if s2[i] > 0.0:
            c = -eta * loss[i] / s2[i]
            m_new[i] = m[i] * np.exp(_clip(c * Gm[i], delta))
            n_new[i] = n[i] * np.exp(_clip(c * Gn[i], delta))
            d_new[i] = d[i] * np.exp(_clip(c * Gd[i], delta))
    return m_new, n_new, d_new
