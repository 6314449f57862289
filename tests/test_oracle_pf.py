"""Pins of the oracle's particle filter (Eq. 9-12, Section 2.2; DA steps
(I)-(V), Section 3.3; perturbation, Section 4.4) against library routines,
closed forms and brute force.  CPU only."""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle


def _case(M, G, seed, spread=0.08):
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.05, 0.6, G)
    y = d[None, :] + rng.normal(0.0, spread, (M, G))
    sigma = rng.uniform(0.03, 0.08, G)
    w0 = rng.dirichlet(np.ones(M))
    return y, d, sigma, w0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weights_match_scipy_gaussian_density(seed):
    """Eq. 9 with diagonal Sigma is scipy's multivariate normal density;
    Eq. 10-11 multiply by the prior weight and normalise."""
    y, d, sigma, w0 = _case(12, 5, seed)
    lik = np.array([multivariate_normal.pdf(d, mean=y[i], cov=np.diag(sigma ** 2))
                    for i in range(len(w0))])
    expect = lik * w0 / (lik * w0).sum()
    w, neff = oracle.pf_weights(y, d, sigma, w0)
    assert np.allclose(w, expect, rtol=1e-12, atol=0)
    assert abs(neff - 1.0 / (expect ** 2).sum()) < 1e-10 * neff


def test_relative_sigma_variant():
    """Section 4.4's Sigma = diag((alpha d_g)^2) with alpha = 0.05."""
    y, d, _, w0 = _case(8, 5, 4, spread=0.01)
    lik = np.array([multivariate_normal.pdf(d, mean=y[i], cov=np.diag((0.05 * d) ** 2))
                    for i in range(8)])
    expect = lik * w0 / (lik * w0).sum()
    w, _ = oracle.pf_weights(y, d, np.ones(5), w0, sigma_rel=0.05)
    assert np.allclose(w, expect, rtol=1e-12, atol=0)


def test_equal_likelihood_keeps_prior_weights_and_neff_bounds():
    M = 10
    y = np.tile(np.array([0.3, 0.1]), (M, 1))
    w0 = np.random.default_rng(3).dirichlet(np.ones(M))
    w, neff = oracle.pf_weights(y, np.array([0.2, 0.2]), np.array([0.05, 0.05]), w0)
    assert np.allclose(w, w0, rtol=1e-14)
    # uniform weights: N_eff = M; a single survivor: N_eff = 1 (Eq. 12)
    _, ne = oracle.pf_weights(y, np.array([0.2, 0.2]), np.array([0.05, 0.05]), np.full(M, 1 / M))
    assert abs(ne - M) < 1e-12
    y2 = y.copy(); y2[4] = [0.2, 0.2]
    w, ne = oracle.pf_weights(y2, np.array([0.2, 0.2]), np.array([1e-3, 1e-3]), np.full(M, 1 / M))
    assert w[4] == 1.0 and ne == 1.0


def test_log_domain_survives_where_direct_product_underflows():
    """Misfits of 60 sigma make every direct likelihood underflow to 0; the
    log-sum-exp form must still return the normalised ratio."""
    M = 4
    d = np.array([0.0])
    y = np.array([[3.0], [3.05], [3.1], [3.2]])
    sigma = np.array([0.05])
    assert np.all(np.exp(-0.5 * ((y[:, 0] - d[0]) / sigma[0]) ** 2) == 0.0)
    w, _ = oracle.pf_weights(y, d, sigma, np.full(M, 0.25))
    chi = -0.5 * ((y[:, 0] - d[0]) / sigma[0]) ** 2
    expect = np.exp(chi - chi.max()) / np.exp(chi - chi.max()).sum()
    assert np.allclose(w, expect, rtol=1e-12)


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8])
def test_systematic_resampling_brute_force(M):
    """For every offset u the counts are floor(M w_i) or ceil(M w_i); over u
    uniform the expected count is exactly M w_i (piecewise-constant in u, so
    a fine midpoint grid integrates it to grid accuracy); the indices equal
    numpy's searchsorted(c, u_j, 'right') on the cumulative weights (particle
    i owns [c_{i-1}, c_i))."""
    rng = np.random.default_rng(M)
    for trial in range(20):
        w = rng.dirichlet(np.ones(M) * (0.3 if trial % 2 else 3.0))
        c = np.cumsum(w); c[-1] = 1.0
        grid = (np.arange(4000) + 0.5) / 4000
        mean_counts = np.zeros(M)
        for u in grid:
            idx = oracle.resample_systematic(w, u)
            assert np.all(np.diff(idx) >= 0)
            uj = (u + np.arange(M)) / M
            assert np.array_equal(idx, np.searchsorted(c, uj, side="right"))
            k = np.bincount(idx, minlength=M)
            assert np.all((k == np.floor(M * w)) | (k == np.ceil(M * w)))
            mean_counts += k
        mean_counts /= len(grid)
        assert np.allclose(mean_counts, M * w, atol=2.0 * M / len(grid))


def test_one_hot_weights_select_one_particle():
    w = np.zeros(7); w[5] = 1.0
    for u in (0.0, 0.3, 0.999999):
        assert np.all(oracle.resample_systematic(w, u) == 5)
    # zero-weight particles are never drawn, even when u_j hits c_i exactly
    w = np.array([0.0, 0.5, 0.0, 0.5])
    assert oracle.resample_systematic(w, 0.0).tolist() == [1, 1, 3, 3]


def test_slot_assignment_keeps_survivors_in_place():
    rng = np.random.default_rng(9)
    for M in (1, 4, 9, 96):
        for _ in range(30):
            w = rng.dirichlet(np.ones(M) * 0.2)
            idx = oracle.resample_systematic(w, rng.random())
            src = oracle.assign_slots(idx)
            assert sorted(src.tolist()) == sorted(idx.tolist())
            k = np.bincount(idx, minlength=M)
            assert np.all(src[k >= 1] == np.nonzero(k >= 1)[0])
            moved = np.nonzero(src != np.arange(M))[0]
            assert len(moved) == int((k == 0).sum())
            assert np.all(np.diff(src[moved]) >= 0)


def test_assimilate_replaces_states_and_perturbs_rain():
    p = oracle.Params(ny=3, nx=4)
    ens = oracle.Ensemble(p, 5)
    for m in range(5):
        ens.h[m] = m + 1.0
        ens.qx[m] = 10.0 * m
    y = np.array([[0.0], [1.0], [2.0], [3.0], [4.0]])
    d = np.array([3.0])
    rain = np.arange(1.0, 6.0); scale = np.linspace(0.6, 1.4, 5)
    beta = np.array([1.01, 0.99, 1.0, 1.02, 0.98])
    w, neff, idx, rm, sc = oracle.pf_assimilate(ens, y, d, np.array([0.4]), rain, scale, 0.37,
                                                beta)
    assert idx is not None and neff < 0.8 * 5
    src = oracle.assign_slots(idx)
    for s in range(5):
        assert np.all(ens.h[s] == src[s] + 1.0)
        assert np.all(ens.qx[s] == 10.0 * src[s])
        assert rm[s] == rain[src[s]] * beta[s]
        assert sc[s] == scale[src[s]]
    assert np.allclose(ens.w, 0.2)
    # above the threshold nothing is resampled and the weights carry over
    ens2 = oracle.Ensemble(p, 5)
    w, neff, idx, _, _ = oracle.pf_assimilate(ens2, y, d, np.array([100.0]), rain, scale, 0.37,
                                              beta)
    assert idx is None and neff > 4.99 and np.allclose(ens2.w, w)
