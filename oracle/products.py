"""FP64 oracle of the ensemble products (test infrastructure only; the
library never imports it).

Section 4.4 (Figs. 15-16) summarises the ensemble by the probability that a
cell's maximum water depth reaches a threshold (20 cm there) and by
percentiles of the depth distribution over the ensemble.  With particle
weights w_i (Eq. 11; equal after a resampling) and each member's maximum
depth over the run hmax_i, per cell:

* exceedance: P = sum_i w_i [hmax_i >= threshold];
* a-percentile: the inverse of the weighted empirical distribution function,
  h_a = min { hmax_i : W_i >= a } with W_i = sum_{j : hmax_j <= hmax_i} w_j,
  and the largest hmax_i if rounding leaves every W_i below a.

Depths and the threshold are compared as FP32 (the stored precision); the
weight sums run in FP64 over the members in index order.
"""
from __future__ import annotations

import numpy as np


def running_max(hmax, h):
    """One step of the running maximum: max(hmax, h) elementwise."""
    return np.maximum(hmax, h)


def exceedance(hmax, w, threshold):
    hm = np.asarray(hmax, np.float32)
    th = np.float32(threshold)
    w = np.asarray(w, np.float64)
    acc = np.zeros(hm.shape[1:])
    for i in range(hm.shape[0]):
        acc = acc + np.where(hm[i] >= th, w[i], 0.0)
    return acc


def weighted_cdf_at_members(hmax, w):
    """W_i per cell: the weight of the members whose value is <= member i's."""
    hm = np.asarray(hmax, np.float32)
    w = np.asarray(w, np.float64)
    M = hm.shape[0]
    W = np.zeros(hm.shape)
    for i in range(M):
        acc = np.zeros(hm.shape[1:])
        for j in range(M):
            acc = acc + np.where(hm[j] <= hm[i], w[j], 0.0)
        W[i] = acc
    return W


def percentiles(hmax, w, levels):
    hm = np.asarray(hmax, np.float32)
    W = weighted_cdf_at_members(hm, w)
    top = hm.max(axis=0)
    out = []
    for a in levels:
        cand = np.where(W >= a, hm.astype(np.float64), np.inf).min(axis=0)
        out.append(np.where(np.isinf(cand), top, cand).astype(np.float32))
    return np.array(out)
