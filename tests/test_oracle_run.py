"""Pins of whole oracle PA runs: invariants, Eq. (Q) at the first step and the
free-energy estimator (Eq. free-energy-estimator) against exact results."""
import math

import numpy as np
import pytest

from oracle import exact

MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST = 0, 1, 2, 3, 4


def _run(oracle, d, L, J, R, nsteps, bf, theta, method, seed, R_cap=0):
    betas = np.linspace(0.0, bf, nsteps + 1)
    run = oracle.Run(d, L, J, R, betas, np.full(nsteps, theta, np.uint32), method, seed,
                     R_cap=R_cap)
    return run, betas


@pytest.mark.parametrize("method", [MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST])
def test_run_invariants(oracle, method):
    d, L = 2, 6
    J = oracle.ferro_couplings(d, L)
    R = 300
    run, betas = _run(oracle, d, L, J, R, 12, 0.6, 2, method, 4, R_cap=2 * R)
    for i in range(12):
        assert run.step() == 0
        sp, E, fam = run.spins(), run.energies(), run.families()
        Ri = run.size
        assert len(E) == Ri and sp.shape == (Ri, L * L)
        for j in range(0, Ri, 23):
            assert oracle.energy(d, L, J, sp[j]) == E[j]
        assert np.all(np.diff(fam.astype(np.int64)) >= 0)     # families stay in order
        c = np.bincount(fam, minlength=R)
        o = run.obs()
        assert o["R_i"] == Ri and int(c.sum()) == Ri
        assert o["sumC2"] == int((c.astype(np.int64) ** 2).sum())
        rho = o["sumC2"] / Ri
        assert 1.0 <= rho <= Ri
        assert o["sumE"] == int(E.astype(np.int64).sum())
        M = sp.astype(np.int64).sum(axis=1)
        assert o["sumAbsM"] == int(np.abs(M).sum()) and o["sumM2"] == int((M * M).sum())
        counts = run.counts()
        anc = run.ancestors()[:Ri]
        assert int(counts.sum()) == Ri
        assert np.array_equal(anc, np.repeat(np.arange(len(counts)), counts))
        if method in (MULTINOMIAL, SYSTEMATIC, RESIDUAL):
            assert Ri == R


def test_first_step_Q_is_ratio_of_partition_functions(oracle):
    """At beta_0 = 0 the population is an exact sample, so E[Q_1] = Z(beta_1)/Z(0)."""
    d, L = 2, 4
    J = oracle.ferro_couplings(d, L)
    E_all, M_all = exact.brute_force(d, L)
    b1 = 0.3
    ref = exact.exact_thermo(E_all, M_all, b1, 16)["lnZ"] - 16 * math.log(2)
    qs = []
    for seed in range(1, 41):
        run, _ = _run(oracle, d, L, J, 500, 1, b1, 1, SYSTEMATIC, seed)
        run.step()
        qs.append(math.exp(run.obs()["lnQ"]))
    qs = np.array(qs)
    assert abs(qs.mean() - math.exp(ref)) < 5 * qs.std(ddof=1) / math.sqrt(len(qs))


@pytest.mark.parametrize("method", [SYSTEMATIC, NEAREST, MULTINOMIAL])
def test_free_energy_estimator_small_lattice(oracle, method):
    """-beta F = N ln2 + sum ln Q reproduces ln Z of the 4x4 Ising model (enumeration)."""
    d, L, bf = 2, 4, 1.0
    J = oracle.ferro_couplings(d, L)
    E_all, M_all = exact.brute_force(d, L)
    th = exact.exact_thermo(E_all, M_all, bf, 16)
    vals, es = [], []
    for seed in range(1, 9):
        run, _ = _run(oracle, d, L, J, 1000, 40, bf, 4, method, seed, R_cap=1500)
        for _ in range(40):
            assert run.step() == 0
        vals.append(run.minus_beta_F())
        es.append(run.obs()["sumE"] / run.size)
    vals = np.array(vals)
    assert abs(vals.mean() - th["lnZ"]) < max(5 * vals.std(ddof=1) / math.sqrt(8), 0.01)
    assert abs(np.mean(es) - th["E"]) < 0.2


def test_free_energy_3d_spin_glass(oracle):
    """3D EA +-J, L=2 (enumeration): the estimator is exact in expectation."""
    d, L, bf = 3, 2, 2.0
    J = oracle.disorder(d, L, 3, 5)
    E_all, M_all = exact.brute_force(d, L, J)
    lnZ = exact.exact_thermo(E_all, M_all, bf, 8)["lnZ"]
    vals = []
    for seed in range(1, 9):
        run, _ = _run(oracle, d, L, J, 800, 30, bf, 3, SYSTEMATIC, seed)
        for _ in range(30):
            assert run.step() == 0
        vals.append(run.minus_beta_F())
    vals = np.array(vals)
    assert abs(vals.mean() - lnZ) < max(5 * vals.std(ddof=1) / math.sqrt(8), 0.01)


@pytest.mark.slow
def test_free_energy_L16_against_kaufman(oracle):
    """2D Ising L=16, R=1000, 100 steps to beta=1, theta=10 (the small reference workload):
    the estimator lands within a few statistical errors of Kaufman's exact ln Z."""
    pytest.importorskip("mpmath")
    L = 16
    J = oracle.ferro_couplings(2, L)
    run, _ = _run(oracle, 2, L, J, 1000, 100, 1.0, 10, NEAREST, 1, R_cap=2000)
    for _ in range(100):
        assert run.step() == 0
    exact_lnZ = exact.kaufman_lnZ(L, 1.0)
    per_spin = (run.minus_beta_F() - exact_lnZ) / (L * L)
    assert abs(per_spin) < 2e-3


def test_checkpoint_free_determinism(oracle):
    """Counter-based RNG: two runs with the same arguments agree bit for bit."""
    d, L = 2, 8
    J = oracle.ferro_couplings(d, L)
    a, _ = _run(oracle, d, L, J, 200, 5, 0.5, 2, POISSON, 8, R_cap=400)
    b, _ = _run(oracle, d, L, J, 200, 5, 0.5, 2, POISSON, 8, R_cap=400)
    for _ in range(5):
        a.step(); b.step()
    assert np.array_equal(a.spins(), b.spins()) and a.obs() == b.obs()


def test_openmp_build_gives_the_same_run(oracle):
    """The multi-core build (replica loop of the sweeps shared among host cores)
    reproduces the single-thread run bit for bit."""
    J = oracle.disorder(3, 4, 3, 1)
    betas = np.linspace(0.0, 2.0, 7)
    th = np.full(6, 3, np.uint32)
    a = oracle.Run(3, 4, J, 300, betas, th, oracle.POISSON, 8, R_cap=600)
    b = oracle.Run(3, 4, J, 300, betas, th, oracle.POISSON, 8, R_cap=600, parallel=True)
    for _ in range(6):
        assert a.step() == 0 and b.step() == 0
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.families(), b.families())
        assert a.obs() == b.obs()
