"""Pins of the exact reference results (Kaufman, transfer matrix, enumeration, Onsager).

These are independent methods: agreement between them pins each one.
"""
import math

import numpy as np
import pytest

from oracle import exact

pytest.importorskip("mpmath")


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("beta", [0.05, 0.3, 0.44068, 0.7, 1.0, 2.0])
def test_kaufman_equals_enumeration(L, beta):
    E, M = exact.brute_force(2, L)
    bf = exact.exact_thermo(E, M, beta, L * L)["lnZ"]
    assert abs(exact.kaufman_lnZ(L, beta) - bf) < 1e-12 * abs(bf)


@pytest.mark.parametrize("L", [4, 6, 8])
@pytest.mark.parametrize("beta", [0.2, 0.44068, 0.9])
def test_kaufman_equals_transfer_matrix(L, beta):
    tm = exact.transfer_lnZ(L, beta)
    assert abs(exact.kaufman_lnZ(L, beta) - tm) < 1e-11 * abs(tm)


def test_kaufman_limits():
    # beta = 0: Z = 2^N
    assert exact.kaufman_lnZ(16, 0.0) == pytest.approx(256 * math.log(2), rel=1e-15)
    assert exact.kaufman_lnZ(16, 1e-9) == pytest.approx(256 * math.log(2), rel=1e-12)
    # beta -> infinity: two ground states of energy -2N
    L, b = 8, 12.0
    assert exact.kaufman_lnZ(L, b) == pytest.approx(2 * L * L * b + math.log(2), rel=1e-12)


@pytest.mark.parametrize("beta,ordered", [(0.3, False), (0.6, True), (1.0, True)])
def test_kaufman_approaches_onsager(beta, ordered):
    L = 96
    per_spin = exact.kaufman_lnZ(L, beta) / (L * L)
    if ordered:  # the periodic lattice keeps both magnetised states: + ln2 / N
        per_spin -= math.log(2) / (L * L)
    assert abs(per_spin - exact.onsager_minus_beta_f(beta)) < 1e-9


def test_enumeration_closed_forms():
    E, M = exact.brute_force(2, 4)
    assert E.min() == -32 and E.max() == 32
    assert (E % 4 == 0).all()
    # number of ground states and of states at E = -24 (one flipped spin: 2*16)
    assert (E == -32).sum() == 2
    assert (E == -24).sum() == 32
    # 3D L=2: 8 sites, 24 bonds (each pair counted twice)
    E3, _ = exact.brute_force(3, 2)
    assert E3.min() == -24 and (E3 == -24).sum() == 2


def test_mattis_gauge_preserves_spectrum():
    rng = np.random.default_rng(5)
    d, L = 2, 4
    J = np.ones(d * L ** d, np.int8)
    g = rng.choice([-1, 1], size=L ** d)
    Jg = exact.mattis_gauge(d, L, J, g)
    E0, _ = exact.brute_force(d, L, J)
    E1, _ = exact.brute_force(d, L, Jg)
    assert np.array_equal(np.sort(E0), np.sort(E1))


def test_golden_kaufman_file_is_current():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "kaufman_lnZ.txt")
    rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
    assert len(rows) == 5 * 201
    for L, b, v in rows[::97]:
        assert float(v) == pytest.approx(exact.kaufman_lnZ(int(L), float(b)), rel=1e-15)
