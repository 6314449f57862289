"""Pins of the oracle's ensemble products (exceedance probability and
percentiles of the maximum depth, Section 4.4): numpy's inverse-CDF
quantile for equal weights, a sort-and-accumulate brute force for unequal
weights, one-hot and degenerate cases, and planted mistakes.  CPU only."""
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
    assert np.allclose(P.exceedance(hm, w, 0.2), want, rtol=1e-14, atol=0)


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


PINS = [pin_equal_weights_quantile, pin_weighted_brute_force, pin_exceedance,
        pin_one_hot_and_extremes]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_products_oracle(pin):
    pin(PROD)


MUTATIONS = [
    ("exceedance strictly above", "np.where(hm[i] >= th, w[i], 0.0)", "np.where(hm[i] > th, w[i], 0.0)"),
    ("cdf counts strictly below", "np.where(hm[j] <= hm[i], w[j], 0.0)",
     "np.where(hm[j] < hm[i], w[j], 0.0)"),
    ("level compared strictly", "np.where(W >= a, hm.astype(np.float64), np.inf).min(axis=0)",
     "np.where(W > a, hm.astype(np.float64), np.inf).min(axis=0)"),
    ("largest qualifying value", "np.where(W >= a, hm.astype(np.float64), np.inf).min(axis=0)",
     "np.where(W >= a, hm.astype(np.float64), -np.inf).max(axis=0)"),
    ("weights ignored", "acc = acc + np.where(hm[j] <= hm[i], w[j], 0.0)",
     "acc = acc + np.where(hm[j] <= hm[i], 1.0 / M, 0.0)"),
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
