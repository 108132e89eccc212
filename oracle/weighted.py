"""Weighted averages of repeated PA runs, Sec. 4 of the paper (test infrastructure only).

Inputs are per-run, per-step rows with the population size R_i, the running sum
of ln Q (the free-energy estimator of Eq. free-energy-estimator without its
common ln Z_0), the exact sums of E, E^2, |M|, M^2, the nominal population size R
and the lattice size N.  For one step:

    omega^(m) = R_i^(m) exp(-beta F^(m)) / sum_m R_i^(m) exp(-beta F^(m))   Eq. (weighted-averages)
    W[O] = sum_m omega^(m) O^(m)
    Wvar[c] = beta^2 N (W[e^2] - W[e]^2)                                       Eq. (Wvar_C)
    Wvar[chi] = beta N (W[m^2] - W[|m|]^2)                                     Eq. (Wvar_Chi)

plus the naive weighting sum_m omega c^(m), the plain means, and the combined
free energy ln(sum_m R^(m) Zhat_m / sum_m R^(m)).  Written with math.fsum over
the runs in index order.
"""
from __future__ import annotations

import math


def weighted_row(rows, R_nominal, N, beta):
    """rows: list of dicts (R_i, sum_lnQ, sumE, sumE2, sumAbsM, sumM2), one per run."""
    a = [math.log(r["R_i"]) + r["sum_lnQ"] for r in rows]
    amax = max(a)
    z = [math.exp(x - amax) for x in a]
    S = math.fsum(z)
    w = [x / S for x in z]
    e, e2, am, m2, c, chi = [], [], [], [], [], []
    for r in rows:
        Ri = r["R_i"]
        ei = r["sumE"] / (Ri * N)
        e2i = r["sumE2"] / (Ri * N * N)
        ami = r["sumAbsM"] / (Ri * N)
        m2i = r["sumM2"] / (Ri * N * N)
        e.append(ei)
        e2.append(e2i)
        am.append(ami)
        m2.append(m2i)
        c.append(beta * beta * N * (e2i - ei * ei))
        chi.append(beta * N * (m2i - ami * ami))

    def W(v):
        return math.fsum(wi * vi for wi, vi in zip(w, v))

    We, We2, Wam, Wm2 = W(e), W(e2), W(am), W(m2)
    b = [math.log(Rn) + r["sum_lnQ"] for Rn, r in zip(R_nominal, rows)]
    bmax = max(b)
    lnZ = bmax + math.log(math.fsum(math.exp(x - bmax) for x in b)) - math.log(sum(R_nominal))
    n = len(rows)
    return {"beta": beta, "n_runs": n, "lnZ": lnZ, "minus_beta_F": N * math.log(2) + lnZ,
            "w_max": max(w), "eff_runs": 1.0 / math.fsum(x * x for x in w),
            "e": We, "e2": We2, "absm": Wam, "m2": Wm2,
            "c": beta * beta * N * (We2 - We * We), "chi": beta * N * (Wm2 - Wam * Wam),
            "c_naive": W(c), "chi_naive": W(chi),
            "e_plain": math.fsum(e) / n, "c_plain": math.fsum(c) / n,
            "chi_plain": math.fsum(chi) / n}
