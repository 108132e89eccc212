"""Pins of the oracle's partial resampling (resample only when the effective size
of the reweighted population falls below alpha R; Sec. 3)."""
import math

import numpy as np
import pytest

from oracle import exact
from oracle import oracle as O


def _run(L=4, R=400, n=10, bf=1.0, theta=2, alpha=0.5, rule="systematic", seed=3, d=2, J=None):
    J = O.ferro_couplings(d, L) if J is None else J
    betas = np.linspace(0.0, bf, n + 1)
    cap = R if rule in ("systematic", "multinomial", "residual") else 2 * R + 64
    return O.Run(d, L, J, R, betas, np.full(n, theta, np.uint32), O.RESAMPLERS[rule], seed,
                 R_cap=cap, alpha=alpha), betas


def test_weighted_sums_with_unit_weights_equal_exact_sums():
    r, _ = _run(alpha=1.0, n=6)
    for _ in range(6):
        assert r.step() == 0
        o = r.obs()
        if o["resampled"]:
            assert o["wsum"] == o["R_i"]
            for w, k in (("wE", "sumE"), ("wE2", "sumE2"), ("wAM", "sumAbsM"), ("wM2", "sumM2")):
                assert o[w] == float(o[k])


def test_alpha_zero_is_annealed_importance_sampling():
    """Never resampling: replica j stays in slot j, and sum ln Q telescopes to
    ln((1/R) sum_j prod_i exp(-dbeta_i E_j^(i-1)))."""
    R, n = 300, 8
    r, betas = _run(R=R, n=n, alpha=0.0, bf=0.8)
    logw = np.zeros(R)
    for i in range(1, n + 1):
        E = r.energies().astype(np.float64)
        logw += -(betas[i] - betas[i - 1]) * E
        assert r.step() == 0
        o = r.obs()
        assert o["resampled"] == 0 and o["R_i"] == R
        assert np.array_equal(r.families(), np.arange(R))
    m = logw.max()
    ref = m + math.log(math.fsum(np.exp(logw - m))) - math.log(R)
    assert math.isclose(r.sum_lnQ(), ref, rel_tol=1e-12, abs_tol=1e-12)
    # the weights are the importance weights up to one common factor
    w = r.weights()
    assert np.allclose(w / w.max(), np.exp(logw - m) / np.exp(logw - m).max(), rtol=1e-12)
    assert 0.5 <= w.max() < 1.0


def test_effective_size_of_the_first_step():
    R = 500
    r, betas = _run(R=R, n=3, alpha=0.0)
    E = r.energies().astype(np.float64)
    g = np.exp(-(betas[1] - betas[0]) * (E - E.min()))
    assert r.step() == 0
    ess = g.sum() ** 2 / (g * g).sum()
    assert math.isclose(r.obs()["ess"], ess, rel_tol=1e-12)


def test_trigger_follows_the_threshold():
    R = 400
    seen = {}
    for alpha in (0.0, 0.3, 0.9, 1.0):
        r, _ = _run(R=R, n=12, alpha=alpha, bf=1.5)
        flags, ess = [], []
        for _ in range(12):
            assert r.step() == 0
            o = r.obs()
            flags.append(o["resampled"])
            ess.append(o["ess"])
            assert o["resampled"] == (o["ess"] < alpha * r.prev_size)
        seen[alpha] = sum(flags)
    # alpha = 1 resamples whenever the weights are not all equal (ESS < R_{i-1})
    assert seen[0.0] == 0 and seen[1.0] >= 6
    assert seen[0.0] <= seen[0.3] <= seen[0.9] <= seen[1.0]


@pytest.mark.parametrize("rule", ["systematic", "nearest"])
def test_free_energy_matches_enumeration(rule):
    """2D Ising L = 4: -beta F at beta = 1 from partial resampling (alpha = 0.5),
    mean over 8 seeds within 5 standard errors of the exact value."""
    L, n = 4, 40
    E_all, M_all = exact.brute_force(2, L)
    exact_lnZ = exact.exact_thermo(E_all, M_all, 1.0, L * L)["lnZ"]
    est = []
    for seed in range(1, 9):
        r, _ = _run(L=L, R=2000, n=n, theta=2, alpha=0.5, rule=rule, seed=seed)
        for _ in range(n):
            assert r.step() == 0
        est.append(r.minus_beta_F())
    m, se = float(np.mean(est)), float(np.std(est, ddof=1) / math.sqrt(len(est)))
    assert abs(m - exact_lnZ) < 5 * se + 1e-3
