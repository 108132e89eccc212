"""Overlap distribution of two independent populations of one disorder sample
(the spin-glass observable of Sec. 4, Figs. 6 and 7), written plainly (test
infrastructure only).

For two populations a and b of the same lattice and couplings at one step,
replica j of a is paired with replica j of b (j < min(R_a, R_b)); the pair's
overlap is q = (1/N) sum_s sigma^a_s sigma^b_s.  k = the number of sites where
the two configurations differ, so q = 1 - 2k/N and sum_s sigma sigma' = N - 2k.

* overlap_hist: the number of pairs at each k = 0..N, from the +-1 arrays,
  computed from the definition (sum of products, not a popcount).
* weighted_P: P(k) = sum_p omega_p hist_p[k] / n_p with omega_p proportional to
  (R_a Zhat_a)(R_b Zhat_b): the two populations are independent, so the weight
  of a pair of runs is the product of their weights of Eq. (weighted-averages).
  Sums with math.fsum.
"""
from __future__ import annotations

import math

import numpy as np


def overlap_hist(spins_a, spins_b):
    """spins_*: int8 arrays [R][N] of +-1.  Returns uint32 counts over k = 0..N."""
    a = np.asarray(spins_a, np.int64)
    b = np.asarray(spins_b, np.int64)
    n = min(a.shape[0], b.shape[0])
    N = a.shape[1]
    dot = (a[:n] * b[:n]).sum(axis=1)          # sum_s sigma^a_s sigma^b_s
    k = (N - dot) // 2                          # sites where the two differ
    return np.bincount(k, minlength=N + 1).astype(np.uint32)


def weighted_P(hists, n_pairs, log_weights):
    """hists: list of count arrays over k; n_pairs: pairs per histogram;
    log_weights: ln(R_a Zhat_a) + ln(R_b Zhat_b) per histogram (common constants
    may be dropped).  Returns P(k) as float64."""
    lmax = max(log_weights)
    w = [math.exp(x - lmax) for x in log_weights]
    S = math.fsum(w)
    bins = len(hists[0])
    out = np.zeros(bins)
    for k in range(bins):
        out[k] = math.fsum(w[p] * (float(hists[p][k]) / n_pairs[p]) for p in range(len(hists))) / S
    return out


def q_values(N):
    """q at each k."""
    return 1.0 - 2.0 * np.arange(N + 1) / N
