"""Oracle of the ensemble products (test infrastructure only; the library
never imports it).

Section 4.4 (Figs. 15-16) summarises the ensemble by the probability that a
cell's maximum water depth reaches a threshold (20 cm there) and by
percentiles of the depth distribution over the ensemble.  With particle
weights w_i (Eq. 11; equal after a resampling) and each member's maximum
depth over the run hmax_i, per cell:

* exceedance: P = sum_i w_i [hmax_i >= threshold];
* a-percentile: the inverse of the weighted empirical distribution function,
  h_a = min { hmax_i : W_i >= a } with W_i = sum_{j : hmax_j <= hmax_i} w_j,
  and the largest hmax_i if every W_i stays below a.

The paper fixes no precision for these sums.  Reading: the weights are
rounded once to whole multiples of 2^-60 (to nearest, ties to even; a weight
below 2^-61 counts as zero) and summed exactly as integers, so every
summation order gives the same W_i; W_i >= a is tested as
W_i * 2^60 >= ceil(a * 2^60).  The exceedance map is the exact integer sum
scaled by 2^-60, rounded to FP64 and then stored as FP32.  Depths and the
threshold are compared as FP32 (the stored precision).
"""
from __future__ import annotations

import math

import numpy as np

FIXED_BITS = 60


def quantized_weights(w):
    """u_i = round(w_i * 2^60) as int64 (w_i * 2^60 is exact in FP64;
    round-half-even is numpy's rint).  The weights are normalised, so every
    sum of them stays below 2^62 and int64 sums are exact."""
    w = np.asarray(w, np.float64)
    u = np.rint(w * 2.0 ** FIXED_BITS).astype(np.int64)
    assert int(u.sum()) < 2 ** 62
    return u


def level_threshold(a: float) -> int:
    """The smallest integer W with W * 2^-60 >= a (a * 2^60 is exact)."""
    return int(math.ceil(float(a) * 2.0 ** FIXED_BITS))


def running_max(hmax, h):
    """One step of the running maximum: max(hmax, h) elementwise."""
    return np.maximum(hmax, h)


def exceedance(hmax, w, threshold):
    hm = np.asarray(hmax, np.float32)
    th = np.float32(threshold)
    u = quantized_weights(w)
    acc = np.zeros(hm.shape[1:], np.int64)
    for i in range(hm.shape[0]):
        acc = acc + np.where(hm[i] >= th, u[i], 0)
    return (acc.astype(np.float64) * 2.0 ** -FIXED_BITS).astype(np.float32)


def weighted_cdf_at_members(hmax, w):
    """W_i per cell as exact integers (units of 2^-60): the weight of the
    members whose value is <= member i's."""
    hm = np.asarray(hmax, np.float32)
    u = quantized_weights(w)
    M = hm.shape[0]
    W = np.zeros(hm.shape, np.int64)
    for i in range(M):
        acc = np.zeros(hm.shape[1:], np.int64)
        for j in range(M):
            acc = acc + np.where(hm[j] <= hm[i], u[j], 0)
        W[i] = acc
    return W


def percentiles(hmax, w, levels):
    hm = np.asarray(hmax, np.float32)
    W = weighted_cdf_at_members(hm, w)
    top = hm.max(axis=0)
    out = []
    for a in levels:
        A = level_threshold(a)
        cand = np.where(W >= A, hm.astype(np.float64), np.inf).min(axis=0)
        out.append(np.where(np.isinf(cand), top, cand).astype(np.float32))
    return np.array(out)
