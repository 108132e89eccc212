"""Pins of the oracle's reweighting, Q and copy counts (Sec. 2 step 2, Sec. 3)."""
import math
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST = 0, 1, 2, 3, 4


def _energies(n, seed, spread=40, base=-400):
    rng = np.random.default_rng(seed)
    return (base + 4 * rng.integers(0, spread, size=n)).astype(np.int32)


@pytest.mark.parametrize("dbeta", [1e-4, 0.01, 0.05, 0.3])
def test_lnQ_matches_high_precision_definition(oracle, dbeta):
    """Eq. (Q): Q = (1/R) sum_j exp(-dbeta E_j)."""
    E = _energies(3000, 1)
    res = oracle.resample(E, 3000, dbeta, SYSTEMATIC, 1, 1)
    with mpmath.workdps(40):
        Q = mpmath.fsum(mpmath.exp(-mpmath.mpf(dbeta) * int(e)) for e in E) / len(E)
        ref = float(mpmath.log(Q))
    assert abs(res["lnQ"] - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("Rprev,R", [(3000, 3000), (2900, 3000), (3100, 3000)])
def test_fixed_point_tau_hat(oracle, Rprev, R):
    """f_j = floor(2^40 tau-hat_j), tau-hat = (R/R_{i-1}) tau (Eq. taus)."""
    dbeta = 0.02
    E = _energies(Rprev, 2)
    res = oracle.resample(E, R, dbeta, NEAREST, 1, 1)
    with mpmath.workdps(40):
        w = [mpmath.exp(-mpmath.mpf(dbeta) * int(e)) for e in E]
        Qn = mpmath.fsum(w)
        for j in range(0, Rprev, 97):
            exact_f = mpmath.mpf(2) ** 40 * R * w[j] / Qn
            assert abs(int(res["f"][j]) - exact_f) <= 2


def _tau(res, R):
    f = res["f"].astype(np.float64)
    return f / 2.0 ** 40


@pytest.mark.parametrize("method", [MULTINOMIAL, SYSTEMATIC, RESIDUAL])
def test_fixed_size_methods_keep_R(oracle, method):
    E = _energies(1000, 3)
    for step in range(1, 6):
        res = oracle.resample(E, 1000, 0.05, method, 7, step)
        assert res["status"] == 0
        assert int(res["counts"].sum()) == 1000 == res["R_new"]


def test_nearest_integer_counts_are_floor_or_ceil(oracle):
    E = _energies(2000, 4)
    res = oracle.resample(E, 2000, 0.05, NEAREST, 7, 3)
    f = res["f"]
    lo = (f >> np.uint64(40)).astype(np.int64)
    c = res["counts"].astype(np.int64)
    assert np.all((c == lo) | (c == lo + 1))
    # an exact multiple of 2^40 gets exactly that many copies
    frac = f & np.uint64((1 << 40) - 1)
    assert np.all(c[frac == 0] == lo[frac == 0])


def test_systematic_matches_label_positions(oracle):
    """Systematic resampling (Fig. 2b): labels at (k + U) T/R, k = 0..R-1, counted per
    box [C_{j-1}, C_j) with exact rational arithmetic."""
    n = 300
    E = _energies(n, 5, spread=12)
    step = 4
    res = oracle.resample(E, n, 0.2, SYSTEMATIC, 9, step)
    U = int(oracle.philox([0, 0x20000000 | 1, step, 0], [9, 0])[0])
    f = [int(v) for v in res["f"]]
    T = sum(f)
    C = [int(v) for v in np.cumsum(np.array(f, dtype=object))]
    counts = np.zeros(n, np.int64)
    j = 0
    for k in range(n):
        pos = Fraction(k * 2 ** 32 + U, 2 ** 32) * Fraction(T, n)
        while pos >= C[j]:
            j += 1
        counts[j] += 1
    assert np.array_equal(counts, res["counts"].astype(np.int64))
    tau = np.array(f, dtype=object) * n / T
    for c, t in zip(res["counts"], tau):
        assert math.floor(t) <= int(c) <= math.ceil(t)


def test_multinomial_matches_searchsorted(oracle):
    """Multinomial resampling (Fig. 2a): R iid labels uniform on the weight axis."""
    n = 500
    E = _energies(n, 6)
    step = 2
    res = oracle.resample(E, n, 0.1, MULTINOMIAL, 13, step)
    f = res["f"].astype(object)
    T = int(sum(f))
    C = np.cumsum(res["f"].astype(np.uint64)).astype(object)
    counts = np.zeros(n, np.int64)
    for k in range(n):
        x = oracle.philox([k >> 1, 0x20000000 | 2, step, 0], [13, 0])
        u = (int(x[3]) << 32 | int(x[2])) if k & 1 else (int(x[1]) << 32 | int(x[0]))
        p = (u * T) >> 64
        j = int(np.searchsorted(np.array(C, dtype=np.uint64), np.uint64(p), side="right"))
        counts[j] += 1
    assert np.array_equal(counts, res["counts"].astype(np.int64))


def test_residual_has_deterministic_part(oracle):
    E = _energies(1500, 7)
    res = oracle.resample(E, 1500, 0.08, RESIDUAL, 3, 9)
    floor_tau = (res["f"] >> np.uint64(40)).astype(np.int64)
    assert np.all(res["counts"].astype(np.int64) >= floor_tau)


def _stats(oracle, E, R, dbeta, method, nrep, seed=17):
    allc = np.stack([oracle.resample(E, R, dbeta, method, seed, s)["counts"].astype(np.float64)
                     for s in range(1, nrep + 1)])
    ref = oracle.resample(E, R, dbeta, method, seed, 1)
    return allc, ref


@pytest.mark.parametrize("method", [MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST])
def test_counts_are_unbiased(oracle, method):
    """<r_j> = tau_j (Sec. 3), with the closed-form variance of each scheme."""
    n, nrep, dbeta = 120, 1500, 0.05
    E = _energies(n, 8, spread=20)
    allc, ref = _stats(oracle, E, n, dbeta, method, nrep)
    f = ref["f"].astype(np.float64)
    T = f.sum()
    tau = f / 2.0 ** 40 if method in (POISSON, NEAREST) else f * n / T
    frac = tau - np.floor(tau)
    if method == MULTINOMIAL:
        var = n * (f / T) * (1 - f / T)
    elif method == POISSON:
        var = tau
    elif method in (NEAREST, SYSTEMATIC):
        var = frac * (1 - frac)
    else:
        var = None
    mean = allc.mean(axis=0)
    if var is not None:
        z = (mean - tau) / np.sqrt(np.maximum(var, 1e-12) / nrep)
        assert np.all(np.abs(z[var > 1e-9]) < 5.5)
        assert np.all(np.abs(mean[var <= 1e-9] - tau[var <= 1e-9]) < 1e-6)
        v = allc.var(axis=0)
        big = var > 0.05
        assert np.all(np.abs(v[big] / var[big] - 1) < 0.35)
    else:
        assert np.all(np.abs(mean - tau) < 5.5 * np.sqrt(np.maximum(frac * (1 - frac), 0.05) /
                                                            nrep) + 0.05)


def test_sampling_variance_ordering(oracle):
    """Eq. (sv): nearest-integer ~ systematic < Poisson ~ multinomial (Sec. 3)."""
    n, dbeta = 800, 0.05
    E = _energies(n, 9, spread=20)
    sv = {}
    for m in (MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST):
        vals = []
        for s in range(1, 41):
            r = oracle.resample(E, n, dbeta, m, 5, s)
            tau = r["f"].astype(np.float64) / 2.0 ** 40
            vals.append(((r["counts"] - tau) ** 2).sum() / n)
        sv[m] = np.mean(vals)
    assert sv[NEAREST] < 0.5 * sv[POISSON]
    assert sv[SYSTEMATIC] < 0.5 * sv[MULTINOMIAL]
    assert sv[RESIDUAL] < sv[MULTINOMIAL]
    assert abs(sv[POISSON] - 1) < 0.1 and abs(sv[MULTINOMIAL] - 1) < 0.1


def test_poisson_distribution_including_large_means(oracle):
    """Counts of one replica follow Poisson(tau-hat), also above the chunk size 16."""
    from scipy import stats
    for spread_beta, target in [(0.0, None), (0.9, None)]:
        n = 60
        E = _energies(n, 10, spread=8)
        allc, ref = _stats(oracle, E, n, spread_beta, POISSON, 1500, seed=23)
        lam = ref["f"].astype(np.float64) / 2.0 ** 40
        j = int(np.argmax(lam))
        x = allc[:, j]
        ks = np.arange(0, int(x.max()) + 2)
        p = stats.poisson.pmf(ks, lam[j])
        obs = np.array([(x == k).sum() for k in ks])
        expct = p * len(x)
        keep = expct > 8
        chi2 = (((obs - expct) ** 2 / expct)[keep]).sum()
        dof = max(int(keep.sum()) - 1, 1)
        assert chi2 < dof + 6 * math.sqrt(2 * dof) + 5
    assert lam.max() > 16  # the chunked path was exercised


def test_capacity_overflow_status(oracle):
    """Variable-size schemes report a capacity overflow instead of writing past R_cap."""
    J = oracle.ferro_couplings(2, 4)
    betas = np.linspace(0, 1, 11)
    run = oracle.Run(2, 4, J, 400, betas, np.ones(10, np.uint32), NEAREST, 3, R_cap=400)
    statuses = [run.step() for _ in range(10)]
    assert 4 in statuses
    first = statuses.index(4)
    assert all(s == 4 for s in statuses[first:])
    assert run.size <= 400
