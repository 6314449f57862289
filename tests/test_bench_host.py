"""Host logic of the benchmark's products roofline: the register sort whose
min/max operations the ALU roofline counts is a sorting network, and its
comparator count follows Batcher's closed form where nothing is pruned."""
import numpy as np
import pytest

import bench


def apply_network(pairs, v):
    v = v.copy()
    for lo, hi in pairs:
        a, b = v[..., lo].copy(), v[..., hi].copy()
        v[..., lo], v[..., hi] = np.minimum(a, b), np.maximum(a, b)
    return v


@pytest.mark.parametrize("p", [5, 6, 7])
def test_unpruned_network_count_is_batchers_closed_form(p):
    # Batcher's odd-even merge sort on 2^p keys takes (p^2 - p + 4) 2^(p-2) - 1
    # comparators (Batcher 1968, "Sorting networks and their applications").
    n = 2 ** p
    want = (p * p - p + 4) * 2 ** (p - 2) - 1
    assert len(bench.sort_network(n)) == want
    assert bench.network_minmax(n) == 2 * want


def test_ninety_six_members_prune_to_1056_comparators():
    pairs = bench.sort_network(96)
    assert len(pairs) == 1056
    assert all(0 <= lo < hi < 96 for lo, hi in pairs)


@pytest.mark.parametrize("M", [1, 7, 32, 33, 64, 90, 96, 100, 128])
def test_pruned_network_sorts_padded_members(M):
    pairs = bench.sort_network(M)
    width = 1 + max(hi for _, hi in pairs)
    rng = np.random.default_rng(M)
    # random values with ties, and 0-1 inputs (the 0-1 principle's cases)
    vals = np.round(rng.normal(size=(400, M)), 1)
    bits = rng.integers(0, 2, size=(2000, M)).astype(np.float64)
    for x in (vals, bits):
        pad = np.full((x.shape[0], max(width, M)), np.inf)
        pad[:, :M] = x
        out = apply_network(pairs, pad)
        np.testing.assert_array_equal(out[:, :M], np.sort(x, axis=1))


def test_unsorted_input_is_caught():
    # the check above fails a network with one comparator dropped
    pairs = bench.sort_network(32)[1:]
    rng = np.random.default_rng(0)
    x = rng.integers(0, 2, size=(4000, 32)).astype(np.float64)
    out = apply_network(pairs, x)
    assert not np.array_equal(out, np.sort(x, axis=1))


def test_summary_repeats_the_extension_figures_at_the_end():
    ext = {"adjoint": {"adj_over_fwd": 1.72900268, "config": "x"},
           "land_cover": {"step_kernel_ms": 1.8107496, "without": {"step_kernel_ms": 1.628},
                          "adjoint": {"adj_over_fwd": 2.62}},
           "batched": {"error": "RuntimeError: no device"},
           "products": {"alu_roofline": {"equal_weights": {"frac": True}}}}
    s = bench.extension_summary(ext)
    assert s == {"adj_over_fwd_1024x1024x1_1800s": 1.729,
                 "adj_over_fwd_2000x2000x96_land_cover": 2.62,
                 "land_cover_step_ms": 1.811, "land_cover_step_ms_without": 1.628}
    assert bench.rounded({"a": [0.123456, 2], "b": "c"}) == {"a": [0.1235, 2], "b": "c"}
