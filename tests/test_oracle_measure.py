"""Pins of the oracle's per-step measurements (Sec. 2 step 4): the sampling
variance of Eq. (sv) and the family statistics (rho_t of Eq. (rho_t), the
family entropy).

The oracle computes them inside its run from its internal count and family
arrays.  These tests reach the same quantities by other routes and compare:
  * closed forms: the initial population (every replica its own family), and
    a nearest-integer step whose expected copy numbers are all equal, where the
    sampling variance follows from the population sizes alone;
  * an independent recomputation from the run's public state: the parents'
    energies before the step give tau-hat_j = R exp(-dbeta E_j) / sum_k
    exp(-dbeta E_k) (the definition of Eq. (taus), evaluated in float64 by a
    shifted log-sum-exp, not through the oracle's fixed-point level table), the
    copy numbers come from the gather (how often each parent is an ancestor),
    and the families of the new population give the entropy and rho_t by
    numpy's unique counts.
Plausible slips these catch: normalising the variance by R_i instead of
R_{i-1}, using tau instead of the rescaled tau-hat for the variable-size rules,
skipping one-member families in the entropy, a wrong sign.
"""
import math

import numpy as np
import pytest

MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST = 0, 1, 2, 3, 4


def _run(oracle, d, L, R, betas, thetas, method, seed, couplings=None):
    J = oracle.ferro_couplings(d, L) if couplings is None else couplings
    return oracle.Run(d, L, J, R, np.asarray(betas, np.float64), np.asarray(thetas, np.uint32),
                      method, seed, R_cap=2 * R + 200)


def _family_stats(fam):
    _, c = np.unique(fam, return_counts=True)
    c = c.astype(np.float64)
    n = c.sum()
    p = c / n
    return float(-(p * np.log(p)).sum()), float((c * c).sum() / n), int((c * c).sum())


def test_initial_population_every_replica_its_own_family(oracle):
    """Step 0: R singleton families, so entropy = ln R, rho_t = 1, sum c^2 = R, SV = 0."""
    for R in (1, 7, 333):
        run = _run(oracle, 2, 4, R, [0.0, 0.1], [1], NEAREST, 2)
        o = run.obs()
        assert o["R_i"] == R
        assert o["sumC2"] == R
        assert math.isclose(o["entropy"], math.log(R), rel_tol=0, abs_tol=1e-12)
        assert o["sv"] == 0.0


def test_sampling_variance_closed_form_for_equal_expected_copies(oracle):
    """Nearest-integer rule.  Step 1 (dbeta = 0.03) changes the population size to
    R_1 != R.  Step 2 has dbeta = 1e-13, so every parent's tau-hat is R / R_1 to
    within 1e-9 (tau itself is 1): r_j takes the values a = floor(R/R_1) and a+1,
    with R_2 - a R_1 parents at a+1.  Eq. (sv) over the R_1 parents is then
      SV = [n1 (1 - phi)^2 + (R_1 - n1) phi^2] / R_1,  phi = R/R_1 - a.
    Using tau instead of tau-hat, or R_2 instead of R_1, changes the value by
    more than a percent here."""
    hits = 0
    for seed in range(1, 12):
        R = 1000
        run = _run(oracle, 2, 8, R, [0.0, 0.03, 0.03 + 1e-13], [2, 2], NEAREST, seed)
        assert run.step() == 0
        R1 = run.size
        if abs(R1 - R) < 5:
            continue
        assert run.step() == 0
        R2 = run.size
        assert run.prev_size == R1
        t = R / R1
        a = math.floor(t)
        phi = t - a
        n1 = R2 - a * R1
        assert 0 <= n1 <= R1
        expect = (n1 * (1 - phi) ** 2 + (R1 - n1) * phi ** 2) / R1
        sv = run.obs()["sv"]
        assert math.isclose(sv, expect, rel_tol=1e-7), (seed, R1, R2, sv, expect)
        # the slips named above give clearly different values
        wrong_norm = expect * R1 / R2
        assert abs(wrong_norm - expect) > 1e-3 * expect
        # tau = 1 for every parent: (r - 1)^2 summed
        n_a = R1 - n1
        wrong_tau = (n1 * (a + 1 - 1) ** 2 + n_a * (a - 1) ** 2) / R1
        assert abs(wrong_tau - expect) > 1e-3 * expect
        hits += 1
    assert hits >= 3


def _tau_hat(E, R, dbeta):
    """tau-hat_j = R exp(-dbeta E_j) / sum_k exp(-dbeta E_k) (Eq. taus), float64."""
    x = -dbeta * E.astype(np.float64)
    x -= x.max()
    w = np.exp(x)
    return R * w / w.sum()


@pytest.mark.parametrize("method", [MULTINOMIAL, SYSTEMATIC, RESIDUAL, POISSON, NEAREST])
def test_measure_against_independent_recomputation(oracle, method):
    """SV, entropy and rho_t of the oracle's measure() against the run's state:
    tau-hat from the parents' energies, r_j from the ancestor array, families
    from the new population.  2D Ising L=8, R=600, a few steps each."""
    R, n = 600, 6
    betas = np.linspace(0.0, 0.9, n + 1)
    run = _run(oracle, 2, 8, R, betas, np.full(n, 2), method, 40 + method)
    sizes_differ = False
    for i in range(1, n + 1):
        E_prev = run.energies().copy()
        Rprev = len(E_prev)
        assert run.step() == 0
        o = run.obs()
        anc = run.ancestors()
        r = np.bincount(anc, minlength=Rprev).astype(np.float64)
        assert r.sum() == o["R_i"] == run.size
        tau = _tau_hat(E_prev, R, betas[i] - betas[i - 1])
        sv = float(((r - tau) ** 2).sum() / Rprev)
        assert math.isclose(o["sv"], sv, rel_tol=1e-9, abs_tol=1e-12), (i, o["sv"], sv)
        ent, rho, c2 = _family_stats(run.families())
        assert math.isclose(o["entropy"], ent, rel_tol=1e-12, abs_tol=1e-12), (i, o["entropy"], ent)
        assert o["sumC2"] == c2
        assert math.isclose(o["sumC2"] / o["R_i"], rho, rel_tol=1e-15)
        assert 0.0 <= o["entropy"] <= math.log(o["R_i"]) + 1e-12
        sizes_differ |= o["R_i"] != Rprev
    if method in (POISSON, NEAREST):
        assert sizes_differ  # the R_i vs R_{i-1} distinction was exercised


def test_entropy_counts_singleton_families(oracle):
    """A population with many one-member families: dropping them from -sum p ln p
    would lower the entropy by their share; the recomputation keeps them."""
    R = 400
    betas = [0.0, 0.05]
    run = _run(oracle, 2, 8, R, betas, [1], SYSTEMATIC, 9)
    assert run.step() == 0
    fam = run.families()
    _, c = np.unique(fam, return_counts=True)
    assert (c == 1).sum() > 100
    ent, _, _ = _family_stats(fam)
    p1 = (c[c == 1] / c.sum())
    assert math.isclose(run.obs()["entropy"], ent, rel_tol=1e-12)
    assert (-(p1 * np.log(p1)).sum()) > 1e-2  # their share is not negligible
