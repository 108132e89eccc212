"""Pins of the oracle's energy, initial state and Metropolis sweeps (Sec. 2, steps 1 and 3)."""
import math

import numpy as np
import pytest

from oracle import exact


def test_energy_matches_enumeration(oracle):
    rng = np.random.default_rng(1)
    for d, L in [(2, 4), (3, 2), (2, 2)]:
        N = L ** d
        J = rng.choice(np.array([-1, 1], np.int8), size=d * N)
        E_all, M_all = exact.brute_force(d, L, J)
        for code in rng.integers(0, 1 << N, size=40):
            sig = (1 - 2 * ((int(code) >> np.arange(N)) & 1)).astype(np.int8)
            assert oracle.energy(d, L, J, sig) == E_all[code]


@pytest.mark.parametrize("d,L", [(2, 16), (2, 6), (3, 4), (3, 6)])
def test_energy_closed_forms(oracle, d, L):
    N = L ** d
    J = oracle.ferro_couplings(d, L)
    assert oracle.energy(d, L, J, np.ones(N, np.int8)) == -d * N
    idx = np.arange(N)
    parity = sum((idx // L ** a) % L for a in range(d)) % 2
    neel = (1 - 2 * parity).astype(np.int8)
    assert oracle.energy(d, L, J, neel) == d * N
    # antiferromagnetic couplings map the Neel state to the ground state
    assert oracle.energy(d, L, -J, neel) == -d * N


def test_disorder_is_balanced_pm1(oracle):
    J = oracle.disorder(3, 8, 3, 0)
    assert set(np.unique(J)) == {-1, 1}
    n = len(J)
    assert abs((J == 1).mean() - 0.5) < 5 * math.sqrt(0.25 / n)
    assert not np.array_equal(J, oracle.disorder(3, 8, 3, 1))
    assert np.array_equal(J, oracle.disorder(3, 8, 3, 0))


def test_initial_state_is_exact_sample_at_beta0(oracle):
    """At beta_0 = 0 the energy histogram of the initial population is g(E) / 2^N."""
    d, L = 2, 4
    E_all, _ = exact.brute_force(d, L)
    levels, g = np.unique(E_all, return_counts=True)
    J = oracle.ferro_couplings(d, L)
    n = 20000
    Es = np.array([oracle.energy(d, L, J, oracle.init_replica(d, L, 11, j)) for j in range(n)])
    obs = np.array([(Es == e).sum() for e in levels])
    expct = n * g / g.sum()
    keep = expct > 5
    chi2 = (((obs - expct) ** 2 / expct)[keep]).sum()
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_thresholds(oracle):
    for beta in [1e-3, 0.1, 0.44068, 1.0, 3.0]:
        t = oracle.thresholds(beta)
        for k in (1, 2, 3):
            exact_t = 2.0 ** 32 * math.exp(-4 * k * beta)
            assert exact_t - 1 <= float(t[k]) <= exact_t
        assert t[1] >= t[2] >= t[3]
    assert oracle.thresholds(0.0)[1] == 0xFFFFFFFF


def _chain_energies(oracle, d, L, J, beta, n, theta, seed):
    sig = oracle.init_replica(d, L, seed, 0)
    out = np.empty(n, np.int64)
    for i in range(n):
        sig, E, _ = oracle.sweeps(d, L, J, sig, seed, i + 1, 0, theta, beta)
        out[i] = E
    return out


@pytest.mark.parametrize("d,L,beta,ea", [(2, 4, 0.4, False), (2, 4, 0.25, True),
                                         (3, 2, 0.5, True)])
def test_metropolis_samples_boltzmann(oracle, d, L, beta, ea):
    """Detailed balance: a long single-replica chain reproduces exp(-beta E)/Z."""
    N = L ** d
    J = oracle.disorder(d, L, 9, 1) if ea else oracle.ferro_couplings(d, L)
    E_all, _ = exact.brute_force(d, L, J)
    levels, g = np.unique(E_all, return_counts=True)
    logw = np.log(g) - beta * levels
    p = np.exp(logw - logw.max())
    p /= p.sum()
    n = 12000
    Es = _chain_energies(oracle, d, L, J, beta, n, 3, 21)
    obs = np.array([(Es == e).sum() for e in levels])
    expct = n * p
    keep = expct > 10
    # allow for residual autocorrelation between samples (factor 2 inflation)
    chi2 = (((obs - expct) ** 2 / expct)[keep]).sum() / 2.0
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 5
    mean_exact = (p * levels).sum()
    sd = math.sqrt((p * (levels - mean_exact) ** 2).sum())
    assert abs(Es.mean() - mean_exact) < 6 * sd / math.sqrt(n / 3)


def test_sweeps_track_energy_and_accepts(oracle):
    d, L = 3, 4
    J = oracle.disorder(d, L, 3, 2)
    sig = oracle.init_replica(d, L, 5, 0)
    s2, E2, acc = oracle.sweeps(d, L, J, sig, 5, 1, 0, 4, 0.7)
    assert E2 == oracle.energy(d, L, J, s2)
    flips = int((s2 != sig).sum())
    assert acc >= flips and (acc - flips) % 2 == 0


def test_mattis_gauge_identity(oracle):
    """The gauge sigma -> g sigma, J -> g J g leaves dE and hence every Metropolis
    decision unchanged: sweeping the gauged system gives the gauged result bit for bit."""
    rng = np.random.default_rng(3)
    for d, L in [(2, 8), (3, 4)]:
        N = L ** d
        J = oracle.ferro_couplings(d, L)
        g = rng.choice(np.array([-1, 1], np.int8), size=N)
        Jg = exact.mattis_gauge(d, L, J, g)
        sig = oracle.init_replica(d, L, 2, 7)
        a, Ea, acc_a = oracle.sweeps(d, L, J, sig, 2, 3, 7, 5, 0.5)
        b, Eb, acc_b = oracle.sweeps(d, L, Jg, (g * sig).astype(np.int8), 2, 3, 7, 5, 0.5)
        assert np.array_equal((g * a).astype(np.int8), b)
        assert Ea == Eb and acc_a == acc_b
