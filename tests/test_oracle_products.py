"""Pins of the oracle's ensemble products (exceedance probability and
percentiles of the maximum depth, Section 4.4): numpy's inverse-CDF
quantile for equal weights, a sort-and-accumulate brute force for unequal
weights, one-hot and degenerate cases, the fixed-point rounding of the
weights and levels, independence of the member order, and planted mistakes.
CPU only."""
import os
import types

import numpy as np
import pytest

from oracle import products as PROD


def pin_equal_weights_quantile(P):
    rng = np.random.default_rng(0)
    hm = rng.random((7, 5, 6)).astype(np.float32)
    levels = (0.1, 0.5, 0.9)            # 7 * a is never an integer: no ties of the CDF
    got = P.percentiles(hm, np.full(7, 1 / 7), levels)
    for k, a in enumerate(levels):
        assert np.array_equal(got[k], np.quantile(hm, a, axis=0, method="inverted_cdf"))


def pin_weighted_brute_force(P):
    rng = np.random.default_rng(1)
    M = 9
    hm = rng.random((M, 4, 3)).astype(np.float32)
    w = rng.random(M)
    w /= w.sum()
    levels = rng.uniform(0.05, 0.95, 5)
    got = P.percentiles(hm, w, levels)
    for r in range(4):
        for c in range(3):
            order = np.argsort(hm[:, r, c], kind="stable")
            cum = np.cumsum(w[order])
            for k, a in enumerate(levels):
                want = hm[order[np.searchsorted(cum, a - 1e-12)], r, c]
                assert got[k, r, c] == want


def pin_exceedance(P):
    rng = np.random.default_rng(2)
    hm = rng.uniform(0, 0.4, (8, 6, 5)).astype(np.float32)
    p = P.exceedance(hm, np.full(8, 0.125), 0.2)
    assert np.array_equal(p, (hm >= np.float32(0.2)).sum(axis=0) * 0.125)
    hm[3, 0, 0] = np.float32(0.2)          # exactly at the threshold counts
    assert P.exceedance(hm, np.full(8, 0.125), 0.2)[0, 0] >= 0.125
    w = rng.random(8); w /= w.sum()
    want = np.array([[w[(hm[:, r, c] >= np.float32(0.2))].sum() for c in range(5)] for r in range(6)])
    got = P.exceedance(hm, w, 0.2)
    assert got.dtype == np.float32
    assert np.allclose(got, want, rtol=1.2e-7, atol=0)   # FP32 rounding of the map


def pin_one_hot_and_extremes(P):
    rng = np.random.default_rng(3)
    hm = rng.random((5, 3, 4)).astype(np.float32)
    w = np.zeros(5); w[2] = 1.0
    got = P.percentiles(hm, w, (0.01, 0.5, 1.0))
    for k in range(3):
        assert np.array_equal(got[k], hm[2])
    eq = np.full(5, 0.2)
    lo, hi = P.percentiles(hm, eq, (1e-9, 1.0))
    assert np.array_equal(lo, hm.min(axis=0)) and np.array_equal(hi, hm.max(axis=0))
    # ties: a cell where every member has the same value
    hm[:, 0, 0] = 0.3
    assert np.all(P.percentiles(hm, eq, (0.1, 0.9))[:, 0, 0] == np.float32(0.3))


def pin_fixed_point_rounding_and_level(P):
    """Weights count in whole units of 2^-60, rounded to nearest; a level a is
    reached when W * 2^-60 >= a.  w_0 = (2^50 + 0.75) 2^-60 counts as
    2^50 + 1 units: the level (2^50 + 1) 2^-60 is reached by member 0 alone
    (truncating the weight would miss it), the level (2^50 + 1.5) 2^-60 is
    not (rounding the level down would reach it)."""
    w0 = (2.0 ** 50 + 0.75) * 2.0 ** -60
    w = np.array([w0, 1.0 - w0])
    hm = np.array([0.1, 0.7], np.float32).reshape(2, 1, 1)
    lo = (2.0 ** 50 + 1.0) * 2.0 ** -60
    hi = (2.0 ** 50 + 1.5) * 2.0 ** -60
    got = P.percentiles(hm, w, (lo, hi))[:, 0, 0]
    assert got[0] == np.float32(0.1) and got[1] == np.float32(0.7)
    assert P.exceedance(hm, w, 0.05)[0, 0] == np.float32(1.0)


def pin_sums_do_not_depend_on_member_order(P):
    """The weighted sums are exact, so relabelling the members changes no
    map, bit for bit."""
    rng = np.random.default_rng(4)
    M = 11
    hm = rng.random((M, 5, 4)).astype(np.float32)
    hm[:4, 0, 0] = np.float32(0.25)              # a tie group
    w = rng.random(M) ** 4; w /= w.sum()
    levels = rng.uniform(0.02, 0.98, 6)
    perm = rng.permutation(M)
    assert np.array_equal(P.percentiles(hm, w, levels), P.percentiles(hm[perm], w[perm], levels))
    assert np.array_equal(P.exceedance(hm, w, 0.5), P.exceedance(hm[perm], w[perm], 0.5))


PINS = [pin_equal_weights_quantile, pin_weighted_brute_force, pin_exceedance,
        pin_one_hot_and_extremes, pin_fixed_point_rounding_and_level,
        pin_sums_do_not_depend_on_member_order]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_products_oracle(pin):
    pin(PROD)


MUTATIONS = [
    ("exceedance strictly above", "np.where(hm[i] >= th, u[i], 0)", "np.where(hm[i] > th, u[i], 0)"),
    ("cdf counts strictly below", "np.where(hm[j] <= hm[i], u[j], 0)",
     "np.where(hm[j] < hm[i], u[j], 0)"),
    ("level compared strictly", "np.where(W >= A, hm.astype(np.float64), np.inf).min(axis=0)",
     "np.where(W > A, hm.astype(np.float64), np.inf).min(axis=0)"),
    ("largest qualifying value", "np.where(W >= A, hm.astype(np.float64), np.inf).min(axis=0)",
     "np.where(W >= A, hm.astype(np.float64), -np.inf).max(axis=0)"),
    ("weights ignored", "acc = acc + np.where(hm[j] <= hm[i], u[j], 0)",
     "acc = acc + np.where(hm[j] <= hm[i], u[0], 0)"),
    ("weights truncated", "np.rint(w * 2.0 ** FIXED_BITS)", "np.floor(w * 2.0 ** FIXED_BITS)"),
    ("level rounded down", "math.ceil(float(a) * 2.0 ** FIXED_BITS)",
     "math.floor(float(a) * 2.0 ** FIXED_BITS)"),
    ("exceedance weights by member 0", "acc = acc + np.where(hm[i] >= th, u[i], 0)",
     "acc = acc + np.where(hm[i] >= th, u[0], 0)"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_product_mistakes(name, old, new):
    with open(os.path.join(os.path.dirname(PROD.__file__), "products.py")) as f:
        src = f.read()
    assert src.count(old) == 1, name
    mod = types.ModuleType("products_mutant")
    exec(compile(src.replace(old, new), "products_mutant.py", "exec"), mod.__dict__)
    caught = False
    for pin in PINS:
        try:
            pin(mod)
        except Exception:  # a failed pin, or a crash on valid input
            caught = True
            break
    assert caught, name
