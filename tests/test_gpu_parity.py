"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer state -- spins, energies, families, copy counts, ancestors, R_i and the
exact population sums -- must agree bit for bit after every temperature step.
ln Q and its running sum use the device's and the host's log(), which may differ
by an ulp, so they are compared to 1e-12 relative; the family entropy and the
sampling variance are order-dependent double sums, compared to 1e-9 relative.
"""
import math

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2401_07965_gb300 import pa  # noqa: E402

RTOL_LNQ = 1e-12
RTOL_SUMS = 1e-9
METHODS = ["multinomial", "systematic", "residual", "poisson", "nearest"]


def _couplings(d, L, kind):
    if kind == "ferro":
        return ("ferro",), O.ferro_couplings(d, L)
    if kind == "ea":
        return ("ea", 3, 5), O.disorder(d, L, 3, 5)
    raise ValueError(kind)


def compare_step(gpu, orc, N, where, initial=False):
    go = gpu.observables()
    oo = orc.obs()
    assert go["R_i"] == oo["R_i"] == orc.size, where
    R_i = orc.size
    for k in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumC2", "accepts"):
        assert go[k] == oo[k], (where, k, go[k], oo[k])
    assert math.isclose(go["lnQ"], oo["lnQ"], rel_tol=RTOL_LNQ, abs_tol=1e-15), where
    assert math.isclose(go["sum_lnQ"], oo["sum_lnQ"], rel_tol=RTOL_LNQ, abs_tol=1e-13), where
    assert math.isclose(go["entropy"], oo["entropy"], rel_tol=RTOL_SUMS, abs_tol=1e-12), where
    assert math.isclose(go["sv"], oo["sv"], rel_tol=RTOL_SUMS, abs_tol=1e-15), where
    assert np.array_equal(gpu.energies(), orc.energies()), where
    assert np.array_equal(gpu.families(), orc.families()), where
    assert np.array_equal(gpu.spins_words(), O.pack_spins(orc.spins())), where
    if not initial:
        assert np.array_equal(gpu.counts(), orc.counts()), where
        assert np.array_equal(gpu.ancestors(), orc.ancestors()[:R_i]), where
    M = orc.spins().astype(np.int64).sum(axis=1)
    assert np.array_equal(gpu.magnetisations().astype(np.int64), M), where


def run_parity(d, L, R, nsteps, bf, theta, method, seed, kind="ferro", R_cap=0, check_every=1,
               queue_cap=None):
    cpl, J = _couplings(d, L, kind)
    betas = np.linspace(0.0, bf, nsteps + 1)
    thetas = np.full(nsteps, theta, np.uint32)
    cap = R_cap or pa.default_capacity(R, method)
    gpu = pa.Population(d, L, R, betas, thetas, method, seed, couplings=cpl, R_cap=cap)
    if queue_cap is not None:
        pa.pa_set_sweep_queue(gpu.ctx, queue_cap)
    orc = O.Run(d, L, J, R, betas, thetas, O.RESAMPLERS[method], seed, R_cap=cap)
    N = L ** d
    compare_step(gpu, orc, N, "init", initial=True)
    for i in range(1, nsteps + 1):
        gpu.step(1)
        assert orc.step() == 0
        if i % check_every == 0 or i == nsteps:
            compare_step(gpu, orc, N, f"step {i}")
    mbf, f = gpu.free_energy()
    assert math.isclose(mbf, orc.minus_beta_F(), rel_tol=1e-12)
    gpu.close()
    return mbf


def test_config1_nearest_full_run():
    """2D Ising L=16, R=1000, beta 0 -> 1 in 100 steps, theta=10, nearest-integer, seed 1."""
    run_parity(2, 16, 1000, 100, 1.0, 10, "nearest", 1, check_every=5)


@pytest.mark.parametrize("method", ["multinomial", "systematic", "residual", "poisson"])
def test_config1_other_rules(method):
    """The same workload for the other rules over its first 25 steps (beta up to 0.25)."""
    betas_full = np.linspace(0, 1.0, 101)
    cpl, J = _couplings(2, 16, "ferro")
    n = 25
    R = 1000
    cap = pa.default_capacity(R, method)
    gpu = pa.Population(2, 16, R, betas_full[: n + 1], np.full(n, 10, np.uint32), method, 1,
                        couplings=cpl, R_cap=cap)
    orc = O.Run(2, 16, J, R, betas_full[: n + 1], np.full(n, 10, np.uint32),
                O.RESAMPLERS[method], 1, R_cap=cap)
    for i in range(1, n + 1):
        gpu.step(1)
        assert orc.step() == 0
        if i % 5 == 0:
            compare_step(gpu, orc, 256, f"{method} step {i}")
    gpu.close()


@pytest.mark.parametrize("method", METHODS)
def test_3d_spin_glass_ragged(method):
    """3D EA +-J L=6 (N=216: last word partial), R=333 (last group of 13), beta to 3."""
    run_parity(3, 6, 333, 12, 3.0, 3, method, 11, kind="ea")


@pytest.mark.parametrize("d,L,R,kind", [(2, 6, 70, "ferro"), (2, 10, 100, "ea"),
                                        (3, 4, 257, "ea"), (3, 10, 64, "ferro"),
                                        (2, 2, 40, "ferro"), (3, 2, 33, "ea"),
                                        (2, 32, 96, "ferro"), (2, 4, 1, "ferro"),
                                        (3, 8, 300, "ea"), (3, 12, 45, "ferro"),
                                        (3, 14, 40, "ea"), (3, 16, 70, "ea"),
                                        (2, 16, 70, "ea"), (2, 32, 50, "ea"),
                                        (2, 64, 40, "ea"), (2, 128, 40, "ferro"),
                                        (2, 128, 33, "ea")])
def test_lattice_shapes(d, L, R, kind):
    # a single replica under Poisson resampling dies out with probability 1/e per step
    for method in (("systematic", "poisson") if R > 8 else ("systematic", "nearest")):
        run_parity(d, L, R, 6, 1.5, 2, method, 5, kind=kind)


def test_theta_zero_and_uneven_schedule():
    d, L, R = 2, 8, 200
    betas = np.array([0.0, 0.01, 0.05, 0.3, 0.31, 1.0])
    thetas = np.array([0, 3, 1, 0, 7], np.uint32)
    for method in METHODS:
        cap = pa.default_capacity(R, method)
        gpu = pa.Population(d, L, R, betas, thetas, method, 9, R_cap=cap)
        orc = O.Run(d, L, O.ferro_couplings(d, L), R, betas, thetas, O.RESAMPLERS[method], 9,
                    R_cap=cap)
        for i in range(len(thetas)):
            gpu.step(1)
            assert orc.step() == 0
            compare_step(gpu, orc, 64, f"{method} step {i + 1}")
        gpu.close()


def test_large_steps_trigger_poisson_chunks_and_big_counts():
    """A single huge temperature step concentrates the weight: tau-hat >> 16."""
    d, L, R = 2, 8, 300
    betas = np.array([0.0, 2.0, 4.0])
    thetas = np.array([1, 1], np.uint32)
    for method in METHODS:
        cap = 4 * R
        gpu = pa.Population(d, L, R, betas, thetas, method, 4, R_cap=cap)
        orc = O.Run(d, L, O.ferro_couplings(d, L), R, betas, thetas, O.RESAMPLERS[method], 4,
                    R_cap=cap)
        for i in range(2):
            gpu.step(1)
            st = orc.step()
            assert st == 0
            compare_step(gpu, orc, 64, f"{method} step {i + 1}")
            if i == 0:  # the jump from beta = 0 concentrates the weight
                assert int(orc.counts().max()) > 16
        gpu.close()


def test_capacity_error_is_reported_not_crashing():
    d, L, R = 2, 8, 400
    betas = np.linspace(0, 1, 21)
    gpu = pa.Population(d, L, R, betas, np.ones(20, np.uint32), "nearest", 3, R_cap=R)
    with pytest.raises(pa.PAError) as ei:
        for _ in range(20):
            gpu.step(1)
            gpu.observables()
    assert ei.value.status == pa.PA_ERR_CAPACITY
    with pytest.raises(pa.PAError) as ei2:
        gpu.step(1)
    assert ei2.value.status == pa.PA_ERR_STATE
    gpu.close()


def test_schedule_exhausted():
    gpu = pa.Population(2, 4, 10, np.array([0.0, 0.5]), np.ones(1, np.uint32), "systematic", 1)
    gpu.step(1)
    with pytest.raises(pa.PAError) as ei:
        gpu.step(1)
    assert ei.value.status == pa.PA_ERR_DONE
    gpu.close()


def test_library_owned_and_torch_workspace_agree():
    betas = np.linspace(0, 0.8, 9)
    th = np.full(8, 3, np.uint32)
    a = pa.Population(2, 16, 500, betas, th, "residual", 2, use_torch_memory=True)
    b = pa.Population(2, 16, 500, betas, th, "residual", 2, use_torch_memory=False)
    a.step(8)
    b.step(8)
    assert np.array_equal(a.spins_words(), b.spins_words())
    assert a.observables() == b.observables()
    a.close()
    b.close()


def test_checkpoint_restore_continues_bit_for_bit():
    betas = np.linspace(0, 1.0, 13)
    th = np.full(12, 4, np.uint32)
    for method in ("poisson", "systematic"):
        ref = pa.Population(3, 4, 300, betas, th, method, 8, couplings=("ea", 3, 1))
        ref.step(12)
        a = pa.Population(3, 4, 300, betas, th, method, 8, couplings=("ea", 3, 1))
        a.step(5)
        words, fam = a.spins_words(), a.families()
        s5 = a.observables()["sum_lnQ"]
        a.close()
        b = pa.Population(3, 4, 300, betas, th, method, 8, couplings=("ea", 3, 1))
        pa.pa_set_state(b.ctx, words, fam, len(fam), 5, s5)
        b.step(7)
        assert np.array_equal(b.spins_words(), ref.spins_words())
        assert np.array_equal(b.families(), ref.families())
        assert b.free_energy() == ref.free_energy()
        ref.close()
        b.close()


@pytest.mark.parametrize("d,L,kind", [(2, 64, "ferro"), (3, 6, "ea"), (2, 32, "ea"),
                                      (2, 128, "ferro"), (2, 16, "ea")])
def test_sweep_launch_configuration_does_not_change_results(d, L, kind):
    cpl, J = _couplings(d, L, kind)
    betas = np.linspace(0, 1.0, 5)
    th = np.full(4, 3, np.uint32)
    ref = None
    for t in (64, 128, 256, 512):
        g = pa.Population(d, L, 200, betas, th, "nearest", 6, couplings=cpl, sweep_threads=t)
        assert pa.pa_get_sweep_threads(g.ctx) == t
        g.step(4)
        cur = (g.spins_words(), g.families(), g.observables())
        g.close()
        if ref is None:
            ref = cur
        else:
            assert np.array_equal(cur[0], ref[0]) and np.array_equal(cur[1], ref[1])
            assert cur[2] == ref[2]
    with pytest.raises(pa.PAError):
        g = pa.Population(d, L, 10, betas, th, "nearest", 6, couplings=cpl, sweep_threads=96)


@pytest.mark.parametrize("sides", [(4, 6, 8, 10), (12, 14, 16)])
def test_3d_group_multiple_does_not_change_results(sides):
    """The grouped 3D kernel with its base replica groups per CTA and with twice as many
    (set before the first step, and changed between steps of a running batch): the
    same spins, families and sums.  Contexts without the grouped kernel refuse 2."""
    Rs = (333, 150, 100, 70)
    runs = [{"dim": 3, "L": L, "R": Rs[k], "couplings": ("ea", 3, k)}
            for k, L in enumerate(sides)]
    betas = np.linspace(0, 2.0, 7)
    th = np.full(6, 2, np.uint32)
    out = []
    for mode in ("one", "two", "switch"):
        b = pa.Batch(runs, betas, th, "systematic", 8)
        if mode == "two":
            pa.pa_set_sweep_groups(b.ctx, 2)
            assert pa.pa_get_sweep_groups(b.ctx) == 2
        for k in range(6):
            if mode == "switch":
                pa.pa_set_sweep_groups(b.ctx, 2 if k % 2 else 1)
            b.step(1)
        out.append([(b.spins_words(m), b.array(m, pa.PA_ARRAY_FAMILY), b.observables(m))
                    for m in range(len(runs))])
        b.close()
    for cur in out[1:]:
        for (s0, f0, o0), (s1, f1, o1) in zip(out[0], cur):
            assert np.array_equal(s0, s1) and np.array_equal(f0, f1) and o0 == o1
    g = pa.Population(2, 16, 64, betas, th, "systematic", 3)
    assert pa.pa_get_sweep_groups(g.ctx) == 1
    pa.pa_set_sweep_groups(g.ctx, 1)
    with pytest.raises(pa.PAError):
        pa.pa_set_sweep_groups(g.ctx, 2)
    g.close()


@pytest.mark.parametrize("d,L,kind,R", [(2, 64, "ferro", 70), (2, 32, "ea", 100),
                                        (3, 8, "ea", 130), (3, 12, "ferro", 40)])
def test_steps_across_zero_top_threshold_bits(d, L, kind, R):
    """The sweep kernels leave out the threshold terms of the energy classes whose
    threshold exp(-beta dE) has eight zero top bits (below 1/256) in the two plane
    blocks every site draws.  Steps on both sides of each boundary (2D: dE = 8 at
    beta = ln 256 / 8, dE = 4 at ln 256 / 4; 3D also dE = 12 at ln 256 / 12) must
    equal the oracle bit for bit."""
    cpl, J = _couplings(d, L, kind)
    c = math.log(256.0)
    edges = [c / 12, c / 8, c / 4]
    betas = np.array([0.0, 0.3] + [e + s for e in edges for s in (-0.01, 0.01)] + [2.5])
    thetas = np.full(len(betas) - 1, 2, np.uint32)
    gpu = pa.Population(d, L, R, betas, thetas, "systematic", 17, couplings=cpl)
    orc = O.Run(d, L, J, R, betas, thetas, O.RESAMPLERS["systematic"], 17)
    N = L ** d
    for i in range(len(betas) - 1):
        gpu.step(1)
        assert orc.step() == 0
        compare_step(gpu, orc, N, f"step {i + 1} beta {betas[i + 1]:.3f}")
    gpu.close()


@pytest.mark.parametrize("d,L,R,kind,method,bf,caps", [
    (2, 64, 96, "ferro", "systematic", 1.0, (0, 32)),
    (3, 6, 150, "ea", "poisson", 3.0, (0, 4)),
    (3, 10, 40, "ea", "nearest", 2.0, (0, 16)),
    (2, 10, 60, "ea", "systematic", 1.5, (0, 4))])
def test_sweep_queue_overflow_path(d, L, R, kind, method, bf, caps):
    """The sweep queues the sites still undecided after eight bits of the uniforms
    and finishes them in a second pass; a site that finds the queue full finishes
    at once.  With the queue capped (0: every such site finishes at once; a small
    cap: some of each) the run must still equal the oracle bit for bit at every
    step: 2D Ising L=64 to beta 1, 3D +-J L=6 and L=10 to beta 2-3, 2D +-J L=10 (the
    general kernel of non-power-of-two 2D lattices)."""
    for cap in caps:
        run_parity(d, L, R, 6, bf, 3, method, 29 + cap, kind=kind, queue_cap=cap)
