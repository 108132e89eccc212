"""Batches of runs (one launch per phase for all runs) against the oracle.

Every run of a batch must equal, bit for bit, the oracle run with the same
replica-slot base and run index; graph replay must equal direct launches; the
device-side weighted averages of Sec. 4 must equal the oracle's on the same
per-run sums.
"""
import math

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from oracle.weighted import weighted_row  # noqa: E402
from paper_2401_07965_gb300 import pa  # noqa: E402


def _oracle_runs(batch, seed, rule):
    out = []
    for m, (spec, base) in enumerate(zip(batch.specs, batch.slot_bases())):
        d, L = spec["dim"], spec["L"]
        cpl = spec.get("couplings", ("ferro",))
        J = O.ferro_couplings(d, L) if cpl[0] == "ferro" else O.disorder(d, L, cpl[1], cpl[2])
        cap = spec.get("R_cap") or pa.default_capacity(spec["R"], rule)
        out.append(O.Run(d, L, J, spec["R"], batch.betas, batch.thetas, O.RESAMPLERS[rule], seed,
                         R_cap=cap, slot_base=base, run_id=m))
    return out


def _compare(batch, orcs, where):
    for m, orc in enumerate(orcs):
        g = batch.observables(m)
        o = orc.obs()
        assert g["R_i"] == o["R_i"], (where, m)
        for k in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumC2", "accepts"):
            assert g[k] == o[k], (where, m, k)
        assert math.isclose(g["sum_lnQ"], o["sum_lnQ"], rel_tol=1e-12, abs_tol=1e-13)
        assert np.array_equal(batch.spins_words(m), O.pack_spins(orc.spins())), (where, m)
        assert np.array_equal(batch.array(m, pa.PA_ARRAY_FAMILY), orc.families()), (where, m)


@pytest.mark.parametrize("rule", ["systematic", "poisson", "multinomial"])
def test_uneven_spin_glass_batch_matches_oracle(rule):
    """3D +-J: L = 4, 6, 4 (two realizations), R = 333, 150, 70; beta to 2 in 8 steps."""
    runs = [{"dim": 3, "L": 4, "R": 333, "couplings": ("ea", 3, 0)},
            {"dim": 3, "L": 6, "R": 150, "couplings": ("ea", 3, 1)},
            {"dim": 3, "L": 4, "R": 70, "couplings": ("ea", 3, 2)}]
    betas = np.linspace(0, 2.0, 9)
    thetas = np.full(8, 3, np.uint32)
    b = pa.Batch(runs, betas, thetas, rule, 17)
    orcs = _oracle_runs(b, 17, rule)
    _compare(b, orcs, "init")
    for i in range(8):
        b.step(1)
        for o in orcs:
            assert o.step() == 0
        _compare(b, orcs, f"step {i + 1}")
    b.close()


@pytest.mark.parametrize("sides", [(4, 6, 8, 10), (4, 6, 8, 10, 12)])
def test_3d_batch_of_several_sides_matches_oracle(sides):
    """3D +-J runs of four sides (one launch of the grouped 3D kernel per side, runs of
    one side interleaved with the others in the run table) and of five sides (more than
    the grouped kernel's plan holds: the general kernel takes every run); R ragged
    against each side's replica groups per CTA; beta to 2 in 5 steps, theta = 2."""
    Rs = (333, 150, 70, 45, 40)
    runs = []
    for k, L in enumerate(sides):
        runs.append({"dim": 3, "L": L, "R": Rs[k], "couplings": ("ea", 3, k)})
    runs.append({"dim": 3, "L": sides[0], "R": 97, "couplings": ("ea", 3, 9)})
    betas = np.linspace(0, 2.0, 6)
    thetas = np.full(5, 2, np.uint32)
    b = pa.Batch(runs, betas, thetas, "systematic", 23)
    orcs = _oracle_runs(b, 23, "systematic")
    _compare(b, orcs, "init")
    for i in range(5):
        b.step(1)
        for o in orcs:
            assert o.step() == 0
        _compare(b, orcs, f"step {i + 1}")
    b.close()


@pytest.mark.parametrize("rule", ["systematic", "nearest"])
def test_uneven_2d_batch_matches_oracle(rule):
    """The weighted-averaging batch shape, scaled down: 2D Ising L=32, four runs of
    R=60 and two of R=240 (uneven populations, one ensemble), beta 0 -> 1 in 6 steps,
    theta=3; every run spin by spin against its oracle run after every step."""
    runs = [{"dim": 2, "L": 32, "R": 60, "ensemble": 0} for _ in range(4)]
    runs += [{"dim": 2, "L": 32, "R": 240, "ensemble": 0} for _ in range(2)]
    betas = np.linspace(0, 1.0, 7)
    thetas = np.full(6, 3, np.uint32)
    b = pa.Batch(runs, betas, thetas, rule, 2000)
    orcs = _oracle_runs(b, 2000, rule)
    _compare(b, orcs, "init")
    for i in range(6):
        b.step(1)
        for o in orcs:
            assert o.step() == 0
        _compare(b, orcs, f"step {i + 1}")
        for m, o in enumerate(orcs):
            assert np.array_equal(b.array(m, pa.PA_ARRAY_ENERGY), o.energies()), (i, m)
            assert np.array_equal(b.array(m, pa.PA_ARRAY_COUNTS), o.counts()), (i, m)
    b.close()


def test_graph_replay_equals_direct_launches():
    runs = [{"dim": 2, "L": 16, "R": 300, "ensemble": 0}, {"dim": 2, "L": 16, "R": 200,
                                                            "ensemble": 0}]
    betas = np.linspace(0, 1.0, 11)
    th = np.full(10, 4, np.uint32)
    a = pa.Batch(runs, betas, th, "nearest", 5, graph=True)
    b = pa.Batch(runs, betas, th, "nearest", 5, graph=False)
    a.step(10)
    for _ in range(10):
        b.step(1)
    for m in range(2):
        assert np.array_equal(a.spins_words(m), b.spins_words(m))
        assert a.observables(m) == b.observables(m)
    a.close()
    b.close()


def test_single_run_batch_equals_pa_init():
    betas = np.linspace(0, 1.0, 6)
    th = np.full(5, 3, np.uint32)
    a = pa.Batch([{"dim": 2, "L": 8, "R": 100}], betas, th, "residual", 3)
    b = pa.Population(2, 8, 100, betas, th, "residual", 3)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.spins_words(0), b.spins_words())
    assert a.observables(0) == b.observables()
    a.close()
    b.close()


def test_weighted_averages_match_oracle_reduction():
    """Ensemble 0: 6 runs of R=400 and 2 of R=1200 (2D Ising L=16); ensemble 1: 3 runs."""
    runs = [{"dim": 2, "L": 16, "R": 400, "ensemble": 0} for _ in range(6)]
    runs += [{"dim": 2, "L": 16, "R": 1200, "ensemble": 0} for _ in range(2)]
    runs += [{"dim": 2, "L": 16, "R": 300, "ensemble": 1} for _ in range(3)]
    n = 20
    betas = np.linspace(0, 1.0, n + 1)
    b = pa.Batch(runs, betas, np.full(n, 5, np.uint32), "systematic", 9)
    b.step(n)
    for ens in (0, 1):
        ids = [m for m, r in enumerate(runs) if r["ensemble"] == ens]
        traces = {m: b.trace(m) for m in ids}
        rows = b.weighted(ens)
        assert len(rows) == n + 1
        for i in (0, 1, 7, n):
            ref = weighted_row([traces[m][i] for m in ids], [runs[m]["R"] for m in ids], 256,
                               float(betas[i]))
            got = rows[i]
            assert got["n_runs"] == len(ids)
            for k in ("lnZ", "e", "e2", "absm", "m2", "c", "chi", "c_naive", "chi_naive",
                      "e_plain", "c_plain", "chi_plain", "w_max", "eff_runs"):
                assert math.isclose(got[k], ref[k], rel_tol=1e-11, abs_tol=1e-12), (ens, i, k)
    with pytest.raises(pa.PAError):
        b.weighted(7)
    b.close()


def test_weighted_free_energy_of_many_small_runs_reaches_kaufman():
    """32 runs of R=2000 and 8 of R=8000 (2D Ising L=16, 100 steps to beta=1, theta=10)
    combined by Eq. (weighted-averages): within 2e-4 per spin of Kaufman's value."""
    import os
    L = 16
    runs = [{"dim": 2, "L": L, "R": 2000} for _ in range(32)]
    runs += [{"dim": 2, "L": L, "R": 8000} for _ in range(8)]
    n = 100
    betas = np.linspace(0, 1.0, n + 1)
    b = pa.Batch(runs, betas, np.full(n, 10, np.uint32), "systematic", 21)
    b.step(n)
    rows = b.weighted(0)
    kf = None
    with open(os.path.join(os.path.dirname(__file__), "golden", "kaufman_lnZ.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            l, bb, v = ln.split()
            if int(l) == L and abs(float(bb) - 1.0) < 1e-12:
                kf = float(v)
    est = rows[n]["minus_beta_F"]
    assert abs(est - kf) / (L * L) < 2e-4
    assert 1.0 <= rows[n]["eff_runs"] <= 40.0
    b.close()


def test_weighted_rows_equal_batch_weighted_averages():
    """Runs summarised as rows (as when they ran on other GPUs) and combined by
    pa_weighted_rows give pa_weighted's numbers bit for bit, and the oracle's."""
    runs = [{"dim": 2, "L": 16, "R": 400} for _ in range(5)] + [{"dim": 2, "L": 16, "R": 900}]
    n = 12
    betas = np.linspace(0, 1.0, n + 1)
    b = pa.Batch(runs, betas, np.full(n, 4, np.uint32), "nearest", 19)
    b.step(n)
    rows = [pa.run_row(b.observables(m), runs[m]["R"]) for m in range(len(runs))]
    got = pa.pa_weighted_rows(rows, 256, float(betas[n]), n)
    ref = b.weighted(0)[n]
    for k in ("lnZ", "minus_beta_F", "e", "e2", "absm", "m2", "c", "chi", "c_naive",
              "chi_naive", "e_plain", "c_plain", "chi_plain", "w_max", "eff_runs"):
        assert got[k] == ref[k], k
    assert got["step"] == n and got["n_runs"] == len(runs)
    oref = weighted_row([b.observables(m) for m in range(len(runs))], [r["R"] for r in runs],
                        256, float(betas[n]))
    for k in ("lnZ", "e", "c", "chi"):
        assert math.isclose(got[k], oref[k], rel_tol=1e-11, abs_tol=1e-12), k
    with pytest.raises(pa.PAError):
        pa.pa_weighted_rows([pa.pa_run_row()], 256, 1.0)
    b.close()
