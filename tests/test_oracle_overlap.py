"""Pins of the overlap-distribution oracle (oracle/overlap.py)."""
import math

import numpy as np

from oracle import overlap as OV


def _rand_spins(rng, R, N):
    return (1 - 2 * rng.integers(0, 2, (R, N))).astype(np.int8)


def test_identical_and_opposite_populations():
    rng = np.random.default_rng(1)
    a = _rand_spins(rng, 50, 36)
    h = OV.overlap_hist(a, a)
    assert h[0] == 50 and h.sum() == 50          # q = 1
    h = OV.overlap_hist(a, -a)
    assert h[36] == 50 and h.sum() == 50         # q = -1
    assert OV.q_values(36)[0] == 1.0 and OV.q_values(36)[36] == -1.0


def test_pairs_by_slot_and_symmetry():
    rng = np.random.default_rng(2)
    a, b = _rand_spins(rng, 40, 20), _rand_spins(rng, 25, 20)
    h = OV.overlap_hist(a, b)
    assert h.sum() == 25                         # min(R_a, R_b) pairs
    assert np.array_equal(h, OV.overlap_hist(b, a))
    # slot j pairs with slot j: a hand count of the first pair
    k0 = int(np.sum(a[0] != b[0]))
    assert OV.overlap_hist(a[:1], b[:1])[k0] == 1


def test_all_pairs_of_a_small_lattice_are_binomial():
    """Every pair of the 16 configurations of N = 4 sites: C(4, k) * 16 pairs at k."""
    confs = np.array([[1 - 2 * ((c >> s) & 1) for s in range(4)] for c in range(16)], np.int8)
    total = np.zeros(5, np.int64)
    for i in range(16):
        total += OV.overlap_hist(np.repeat(confs[i:i + 1], 16, 0), confs)
    assert list(total) == [16 * math.comb(4, k) for k in range(5)]


def test_independent_uniform_populations_follow_binomial():
    rng = np.random.default_rng(3)
    N, R = 64, 20000
    h = OV.overlap_hist(_rand_spins(rng, R, N), _rand_spins(rng, R, N))
    pmf = np.array([math.comb(N, k) for k in range(N + 1)], float) / 2.0 ** N
    exp_counts = R * pmf
    m = exp_counts > 5
    chi2 = float(np.sum((h[m] - exp_counts[m]) ** 2 / exp_counts[m]))
    dof = int(m.sum()) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_gauge_transformation_leaves_overlaps_unchanged():
    """A Mattis gauge flip sigma_s -> eps_s sigma_s applied to both populations (they
    are then configurations of the gauge-transformed sample) keeps every overlap."""
    rng = np.random.default_rng(4)
    L = 4
    eps = (1 - 2 * rng.integers(0, 2, L * L)).astype(np.int8)
    a, b = _rand_spins(rng, 30, L * L), _rand_spins(rng, 30, L * L)
    assert np.array_equal(OV.overlap_hist(a, b), OV.overlap_hist(a * eps, b * eps))


def test_weighted_estimate():
    h1 = np.array([2, 6, 2], np.uint32)
    h2 = np.array([0, 4, 4], np.uint32)
    # equal weights: mean of the normalised histograms
    P = OV.weighted_P([h1, h2], [10, 8], [0.0, 0.0])
    assert np.allclose(P, [0.5 * (0.2 + 0.0), 0.5 * (0.6 + 0.5), 0.5 * (0.2 + 0.5)], 0, 1e-15)
    assert math.isclose(P.sum(), 1.0, rel_tol=1e-15)
    # weights e^1 : e^0, and a common constant cancels
    P1 = OV.weighted_P([h1, h2], [10, 8], [1.0, 0.0])
    P2 = OV.weighted_P([h1, h2], [10, 8], [101.0, 100.0])
    w = math.e / (math.e + 1.0)
    assert np.allclose(P1, w * h1 / 10 + (1 - w) * h2 / 8, 0, 1e-15)
    assert np.allclose(P1, P2, 0, 1e-15)
    # one overwhelming weight selects its histogram
    assert np.allclose(OV.weighted_P([h1, h2], [10, 8], [0.0, 800.0]), h2 / 8, 0, 1e-15)
