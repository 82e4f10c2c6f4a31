"""Empirical FDR curve from the permutation histogram of ``krux_permute``.

Section "P-value calculation and empirical FDR correction": the FDR of a
threshold P <= P_c is the average, over the permuted data sets, of the number of
pairs with P' <= P, divided by the number of pairs with P' <= P in the real data.
``krux_permute`` bins every pair with p < P_c by b = floor((-log10 p + log10 P_c) / w);
summing bins b and above counts the pairs with p <= P_c * 10^(-b w), so the curve
is exact at those thresholds.  Host arithmetic on the counts only."""
from __future__ import annotations

import numpy as np


def fdr_curve(hist, pthresh, bin_width):
    """hist: [1 + P, bins] counts (row 0 real data).  Returns dict of arrays over b:
    threshold P_b = P_c * 10^(-b w), n_real (pairs of the real data with p <= P_b),
    mean_perm (mean over permutations of the same count) and fdr = mean_perm / n_real
    (NaN where n_real is 0)."""
    h = np.asarray(hist.cpu() if hasattr(hist, "cpu") else hist, dtype=np.int64)
    if h.ndim != 2 or h.shape[0] < 2:
        raise ValueError("need a [1 + P, bins] histogram with P >= 1")
    tail = np.cumsum(h[:, ::-1], axis=1)[:, ::-1]  # tail[q, b] = sum of bins >= b
    n_real = tail[0]
    mean_perm = tail[1:].mean(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        fdr = np.where(n_real > 0, mean_perm / np.maximum(n_real, 1), np.nan)
    thr = pthresh * 10.0 ** (-bin_width * np.arange(h.shape[1]))
    return dict(threshold=thr, n_real=n_real, mean_perm=mean_perm, fdr=fdr)


def hit_fdr(hit_p, hist, pthresh, bin_width):
    """FDR of each real hit, read off the curve at the largest grid threshold
    P_b >= p (the curve is a step function between grid points)."""
    c = fdr_curve(hist, pthresh, bin_width)
    p = np.asarray(hit_p.cpu() if hasattr(hit_p, "cpu") else hit_p, dtype=np.float64)
    b = np.floor((-np.log10(p) + np.log10(pthresh)) / bin_width).astype(np.int64)
    b = np.clip(b, 0, len(c["fdr"]) - 1)
    return c["fdr"][b]
