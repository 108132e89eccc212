"""Partial resampling on the GPU against the oracle: decisions, effective sizes,
weights, counts, spins and families bit-exact after every step; ln Q within
1e-12; weighted averages within 1e-12."""
import math

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2401_07965_gb300 import pa  # noqa: E402


def _compare(g, o, pop_spins, pop_fam, pop_w, orc, where):
    assert g["R_i"] == o["R_i"], where
    assert g["resampled"] == o["resampled"], where
    assert g["ess"] == o["ess"], where
    for k in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumC2", "accepts"):
        assert g[k] == o[k], (where, k)
    assert math.isclose(g["sum_lnQ"], o["sum_lnQ"], rel_tol=1e-12, abs_tol=1e-13), where
    assert np.array_equal(pop_spins, O.pack_spins(orc.spins())), where
    assert np.array_equal(pop_fam, orc.families()), where
    assert np.array_equal(pop_w, orc.weights()), where
    N = orc.N
    for gk, wk, scale in (("e", "wE", N), ("e2", "wE2", N * N), ("absm", "wAM", N),
                          ("m2", "wM2", N * N)):
        ref = o[wk] / (o["wsum"] * scale)
        assert math.isclose(g[gk], ref, rel_tol=1e-12, abs_tol=1e-15), (where, gk)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("rule", ["systematic", "nearest", "multinomial", "poisson"])
def test_single_run_matches_oracle(rule, alpha):
    d, L, R, n = 2, 8, 300, 12
    betas = np.linspace(0.0, 1.2, n + 1)
    thetas = np.full(n, 2, np.uint32)
    cap = pa.default_capacity(R, rule)
    p = pa.Population(d, L, R, betas, thetas, rule, 31, R_cap=cap)
    p.set_partial_resampling(alpha)
    orc = O.Run(d, L, O.ferro_couplings(d, L), R, betas, thetas, O.RESAMPLERS[rule], 31,
                R_cap=cap, alpha=alpha)
    _compare(p.observables(), orc.obs(), p.spins_words(), p.families(), p.weights(), orc, 0)
    for i in range(n):
        p.step(1)
        assert orc.step() == 0
        _compare(p.observables(), orc.obs(), p.spins_words(), p.families(), p.weights(), orc,
                 i + 1)
    p.close()


def test_spin_glass_batch_matches_oracle():
    """Two runs of uneven size in one batch (3D +-J L = 4), alpha = 0.6, residual rule."""
    runs = [{"dim": 3, "L": 4, "R": 257, "couplings": ("ea", 3, 0)},
            {"dim": 3, "L": 4, "R": 130, "couplings": ("ea", 3, 1)}]
    n = 10
    betas = np.linspace(0.0, 2.0, n + 1)
    thetas = np.full(n, 3, np.uint32)
    b = pa.Batch(runs, betas, thetas, "residual", 8)
    b.set_partial_resampling(0.6)
    orcs = []
    for m, (spec, base) in enumerate(zip(runs, b.slot_bases())):
        J = O.disorder(3, 4, 3, spec["couplings"][2])
        orcs.append(O.Run(3, 4, J, spec["R"], betas, thetas, O.RESAMPLERS["residual"], 8,
                          R_cap=spec["R"], slot_base=base, run_id=m, alpha=0.6))
    for i in range(n):
        b.step(1)
        for m, o in enumerate(orcs):
            assert o.step() == 0
            _compare(b.observables(m), o.obs(), b.spins_words(m),
                     b.array(m, pa.PA_ARRAY_FAMILY), b.array(m, pa.PA_ARRAY_WEIGHT), o,
                     (m, i + 1))
    b.close()


def test_many_blocks_match_oracle():
    """R = 100000 replicas of the 8 x 8 lattice: 49 scan blocks, so the weight sums run
    through the two-level tree; alpha = 0.9, steps of 0.02 (some resample, some do not),
    systematic, one sweep per step."""
    d, L, R, n = 2, 8, 100000, 6
    betas = np.linspace(0.0, 0.12, n + 1)
    thetas = np.full(n, 1, np.uint32)
    p = pa.Population(d, L, R, betas, thetas, "systematic", 4)
    p.set_partial_resampling(0.9)
    orc = O.Run(d, L, O.ferro_couplings(d, L), R, betas, thetas, O.RESAMPLERS["systematic"], 4,
                R_cap=R, alpha=0.9)
    flags = []
    for i in range(n):
        p.step(1)
        assert orc.step() == 0
        g, o = p.observables(), orc.obs()
        flags.append(o["resampled"])
        assert g["resampled"] == o["resampled"] and g["ess"] == o["ess"]
        assert math.isclose(g["sum_lnQ"], o["sum_lnQ"], rel_tol=1e-12)
        assert np.array_equal(p.weights(), orc.weights())
        assert np.array_equal(p.families(), orc.families())
    assert np.array_equal(p.spins_words(), O.pack_spins(orc.spins()))
    assert 0 < sum(flags) < n   # both kinds of step occurred
    p.close()


def test_partial_free_energy_reaches_kaufman():
    """2D Ising L = 16, R = 20000, 100 steps to beta = 1, theta = 10, alpha = 0.5: within
    1e-4 per spin of Kaufman's value, with fewer resampling steps than steps."""
    import os
    L, n = 16, 100
    betas = np.linspace(0.0, 1.0, n + 1)
    p = pa.Population(2, L, 20000, betas, np.full(n, 10, np.uint32), "systematic", 12)
    p.set_partial_resampling(0.5)
    p.step(n)
    kf = None
    with open(os.path.join(os.path.dirname(__file__), "golden", "kaufman_lnZ.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            l, bb, v = ln.split()
            if int(l) == L and abs(float(bb) - 1.0) < 1e-12:
                kf = float(v)
    mbf, _ = p.free_energy()
    assert abs(mbf - kf) / (L * L) < 1e-4
    rows = p.trace()
    assert 0 < sum(r["resampled"] for r in rows[1:]) < n
    p.close()


def test_partial_resampling_arguments():
    betas = np.linspace(0.0, 1.0, 4)
    p = pa.Population(2, 8, 64, betas, np.full(3, 1, np.uint32), "systematic", 1)
    with pytest.raises(pa.PAError):
        p.set_partial_resampling(1.5)
    p.step(1)
    with pytest.raises(pa.PAError):       # only before the first step
        p.set_partial_resampling(0.5)
    p.close()


def test_partial_resampling_under_graph_replay_equals_direct_launches():
    import torch
    runs = [{"dim": 2, "L": 16, "R": 500}, {"dim": 2, "L": 16, "R": 300}]
    betas = np.linspace(0.0, 1.0, 21)
    th = np.full(20, 3, np.uint32)
    a = pa.Batch(runs, betas, th, "nearest", 6, stream=torch.cuda.Stream(), graph=True)
    b = pa.Batch(runs, betas, th, "nearest", 6, graph=False)
    a.set_partial_resampling(0.5)
    b.set_partial_resampling(0.5)
    a.step(20)
    for _ in range(20):
        b.step(1)
    for m in range(2):
        assert np.array_equal(a.spins_words(m), b.spins_words(m))
        assert np.array_equal(a.array(m, pa.PA_ARRAY_WEIGHT), b.array(m, pa.PA_ARRAY_WEIGHT))
        assert a.observables(m) == b.observables(m)
    a.close()
    b.close()
