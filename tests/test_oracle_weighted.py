"""Pins of the weighted averages of Sec. 4 (oracle/weighted.py)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle.weighted import weighted_row

MULTINOMIAL, SYSTEMATIC = 0, 1


def _row(run):
    o = run.obs()
    return {k: o[k] for k in ("R_i", "sum_lnQ", "sumE", "sumE2", "sumAbsM", "sumM2")}


def test_single_run_reduces_to_its_own_estimates():
    rows = [{"R_i": 100, "sum_lnQ": 3.2, "sumE": -5000, "sumE2": 260000, "sumAbsM": 1200,
             "sumM2": 30000}]
    w = weighted_row(rows, [100], 64, 0.5)
    e, e2 = -5000 / (100 * 64), 260000 / (100 * 64 * 64)
    assert w["w_max"] == 1.0 and w["eff_runs"] == 1.0
    assert w["e"] == pytest.approx(e) and w["c"] == pytest.approx(0.25 * 64 * (e2 - e * e))
    assert w["c"] == pytest.approx(w["c_naive"]) and w["lnZ"] == pytest.approx(3.2)


def test_equal_free_energies_give_size_weighted_means():
    """omega ~ R_i when the runs' free-energy estimates agree (closed form of the weights)."""
    rows = [{"R_i": 100, "sum_lnQ": 1.0, "sumE": -640, "sumE2": 5000, "sumAbsM": 0, "sumM2": 0},
            {"R_i": 300, "sum_lnQ": 1.0, "sumE": -3840, "sumE2": 60000, "sumAbsM": 0,
             "sumM2": 0}]
    w = weighted_row(rows, [100, 300], 64, 1.0)
    e1, e2 = -640 / 6400, -3840 / 19200
    assert w["e"] == pytest.approx(0.25 * e1 + 0.75 * e2)
    assert w["eff_runs"] == pytest.approx(1 / (0.25 ** 2 + 0.75 ** 2))
    assert w["lnZ"] == pytest.approx(1.0)


def test_weights_follow_free_energy_differences():
    """Two equal-size runs whose ln Z differ by ln 3 get weights 1/4 and 3/4."""
    rows = [{"R_i": 50, "sum_lnQ": 2.0, "sumE": 100, "sumE2": 1000, "sumAbsM": 10, "sumM2": 40},
            {"R_i": 50, "sum_lnQ": 2.0 + math.log(3), "sumE": 300, "sumE2": 3000,
             "sumAbsM": 30, "sumM2": 80}]
    w = weighted_row(rows, [50, 50], 16, 0.3)
    assert w["w_max"] == pytest.approx(0.75)
    assert w["e"] == pytest.approx(0.25 * 100 / 800 + 0.75 * 300 / 800)
    assert w["lnZ"] == pytest.approx(math.log((math.exp(2) + math.exp(2 + math.log(3))) / 2))


def test_weighted_free_energy_of_oracle_runs_is_exact_in_expectation():
    """Several small oracle runs of the 4x4 Ising model combined by Eq. (weighted-averages)
    give ln Z within the spread of the runs (enumeration)."""
    from oracle import exact
    E_all, M_all = exact.brute_force(2, 4)
    bf, n = 0.8, 20
    betas = np.linspace(0, bf, n + 1)
    runs = []
    for m in range(6):
        r = O.Run(2, 4, O.ferro_couplings(2, 4), 200, betas, np.full(n, 2, np.uint32),
                  SYSTEMATIC, 40 + m)
        for _ in range(n):
            r.step()
        runs.append(r)
    w = weighted_row([_row(r) for r in runs], [200] * 6, 16, bf)
    exact_lnZ = exact.exact_thermo(E_all, M_all, bf, 16)["lnZ"] - 16 * math.log(2)
    spread = np.std([r.obs()["sum_lnQ"] for r in runs])
    assert abs(w["lnZ"] - exact_lnZ) < 4 * spread + 0.01
