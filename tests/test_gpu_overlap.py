"""Overlap distribution of two populations per disorder sample on the GPU against
the oracle: histograms bit-exact, weighted estimate within 1e-12."""
import math

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from oracle import overlap as OV  # noqa: E402
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


def _check(batch, orcs, pairs, N):
    hist, P = batch.overlap(pairs)
    ref_h, n_p, lw = [], [], []
    for a, b in pairs:
        ha = OV.overlap_hist(orcs[a].spins(), orcs[b].spins())
        ref_h.append(ha)
        oa, ob = orcs[a].obs(), orcs[b].obs()
        n_p.append(min(oa["R_i"], ob["R_i"]))
        lw.append(math.log(oa["R_i"]) + oa["sum_lnQ"] + math.log(ob["R_i"]) + ob["sum_lnQ"])
    for p in range(len(pairs)):
        assert np.array_equal(hist[p], ref_h[p]), p
        assert hist[p].sum() == n_p[p]
    ref_P = OV.weighted_P(ref_h, n_p, lw)
    assert np.allclose(P, ref_P, rtol=1e-12, atol=1e-15)
    assert math.isclose(P.sum(), 1.0, rel_tol=1e-12)


@pytest.mark.parametrize("rule,runs", [
    ("systematic", [{"dim": 3, "L": 4, "R": 300, "couplings": ("ea", 3, 0)},
                    {"dim": 3, "L": 4, "R": 300, "couplings": ("ea", 3, 0)},
                    {"dim": 3, "L": 4, "R": 200, "couplings": ("ea", 3, 1)},
                    {"dim": 3, "L": 4, "R": 200, "couplings": ("ea", 3, 1)}]),
    ("poisson", [{"dim": 2, "L": 10, "R": 250, "couplings": ("ea", 3, 7)},
                 {"dim": 2, "L": 10, "R": 250, "couplings": ("ea", 3, 7)}]),
    ("nearest", [{"dim": 3, "L": 10, "R": 90, "couplings": ("ea", 3, 2)},
                 {"dim": 3, "L": 10, "R": 90, "couplings": ("ea", 3, 2)}]),
])
def test_overlap_histograms_match_oracle(rule, runs):
    n = 6
    betas = np.linspace(0.0, 1.5, n + 1)
    thetas = np.full(n, 3, np.uint32)
    b = pa.Batch(runs, betas, thetas, rule, 23)
    orcs = _oracle_runs(b, 23, rule)
    pairs = [(2 * i, 2 * i + 1) for i in range(len(runs) // 2)]
    N = runs[0]["L"] ** runs[0]["dim"]
    _check(b, orcs, pairs, N)             # at beta = 0 (initial populations)
    for _ in range(n):
        b.step(1)
        for o in orcs:
            assert o.step() == 0
    _check(b, orcs, pairs, N)
    if len(pairs) > 1:                     # a run may appear in several pairs
        _check(b, orcs, [(0, 1), (1, 0), (2, 3)], N)
    b.close()


def test_initial_populations_are_binomial_at_full_size():
    """At beta = 0 the populations are iid uniform: k ~ Binomial(N, 1/2) over 10^5 pairs
    (2D L = 32, the lattice of the paper's P(q) figures)."""
    L, R = 32, 100000
    runs = [{"dim": 2, "L": L, "R": R, "couplings": ("ea", 3, 0)} for _ in range(2)]
    b = pa.Batch(runs, np.linspace(0, 1, 3), np.full(2, 1, np.uint32), "systematic", 5)
    hist, P = b.overlap([(0, 1)])
    N = L * L
    k = np.arange(N + 1)
    mean = float((hist[0] * k).sum()) / R
    var = float((hist[0] * (k - mean) ** 2).sum()) / R
    assert abs(mean - N / 2) < 6 * math.sqrt(N / 4 / R)
    assert abs(var / (N / 4) - 1) < 0.03
    assert np.allclose(P, hist[0] / R, rtol=1e-13, atol=0)
    b.close()


def test_overlap_argument_errors():
    runs = [{"dim": 2, "L": 8, "R": 64}, {"dim": 2, "L": 8, "R": 64}, {"dim": 2, "L": 6, "R": 64}]
    b = pa.Batch(runs, np.linspace(0, 1, 3), np.full(2, 1, np.uint32), "systematic", 5)
    with pytest.raises(pa.PAError):
        b.overlap([(0, 0)])                 # a run with itself
    with pytest.raises(pa.PAError):
        b.overlap([(0, 2)])                 # different N
    with pytest.raises(pa.PAError):
        b.overlap([(0, 5)])                 # no such run
    b.close()
