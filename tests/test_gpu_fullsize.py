"""GPU checks at the benchmark's full size and against independent references.

* Full size (2D L=64, R=100000, theta=10, the benchmark's tuned launch
  configuration): after a temperature step, every copy count and ln Q equal
  the oracle's on the GPU's own pre-step energies; the ancestor and family
  arrays follow from the counts; a sample of replicas is swept by the oracle
  from the GPU's pre-step spins and must match bit for bit.
* Philox4x32-10 of the oracle equals cuRAND's Philox generator.
* Accuracy: the free-energy estimator (Eq. free-energy-estimator) reaches
  Kaufman's exact value of the 2D Ising model within 1e-4 per spin.
"""
import ctypes as C
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2401_07965_gb300 import pa, tune  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
RULES = ["multinomial", "systematic", "residual", "poisson", "nearest"]


def _kaufman(L):
    out = {}
    with open(os.path.join(HERE, "golden", "kaufman_lnZ.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            l, b, v = ln.split()
            if int(l) == L:
                out[round(float(b), 6)] = float(v)
    return out


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("k", [2, 149])
def test_full_size_step_against_oracle(rule, k):
    """Step k+1 of the benchmark run: k = 2 (beta = 0.015, few replicas need a
    Metropolis draw) and k = 149 (beta = 0.75, nearly every site needs one and the
    thresholds' top bits are zero)."""
    L, R, theta, seed, n = 64, 100000, 10, 7, 200
    betas = np.linspace(0.0, 1.0, n + 1)
    thetas = np.full(n, theta, np.uint32)
    threads = tune.best_sweep_threads(2, L, R, theta=theta)
    g = pa.Population(2, L, R, betas, thetas, rule, seed, sweep_threads=threads)
    N, W = L * L, (L * L) // 32
    # initial population: sampled replicas against the oracle's exact sampling
    words0 = g.spins_words()
    rng = np.random.default_rng(1)
    for j in rng.choice(R, 16, replace=False):
        assert np.array_equal(words0[j], O.pack_spins(O.init_replica(2, L, seed, int(j))[None])[0])
    g.step(k)
    E_pre, fam_pre, words_pre = g.energies(), g.families(), g.spins_words()
    g.step(1)
    i = k + 1
    obs = g.observables()
    ref = O.resample(E_pre, R, betas[i] - betas[i - 1], O.RESAMPLERS[rule], seed, i)
    assert ref["status"] == 0
    counts = g.counts()
    assert np.array_equal(counts, ref["counts"])
    assert obs["R_i"] == ref["R_new"]
    assert math.isclose(obs["lnQ"], ref["lnQ"], rel_tol=1e-12)
    anc = g.ancestors()
    assert np.array_equal(anc, np.repeat(np.arange(len(counts), dtype=np.uint32), counts))
    fam = g.families()
    assert np.array_equal(fam, fam_pre[anc])
    # family statistics of the new population (families span many scan blocks at
    # this size, late in the run some of them thousands of slots)
    _, c = np.unique(fam, return_counts=True)
    assert obs["sumC2"] == int((c.astype(np.int64) ** 2).sum())
    pf = c / c.sum()
    assert math.isclose(obs["entropy"], float(-(pf * np.log(pf)).sum()), rel_tol=1e-9)
    words, E = g.spins_words(), g.energies()
    J = O.ferro_couplings(2, L)
    for d in rng.choice(obs["R_i"], 12, replace=False):
        parent = words_pre[anc[d]]
        bits = ((parent[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:N]
        sig = (1 - 2 * bits.astype(np.int8)).astype(np.int8)
        s2, E2, _ = O.sweeps(2, L, J, sig, seed, i, int(d), theta, betas[i])
        assert np.array_equal(words[d], O.pack_spins(s2[None])[0]), (rule, d)
        assert E[d] == E2
    g.close()


@pytest.mark.parametrize("rule", ["systematic", "nearest"])
def test_largest_population_step_against_oracle(rule):
    """The largest population the 2^-40 fixed-point weights allow (R and R_cap below 2^24):
    R = 2^24 - 1 for the fixed-size rule; for the nearest-integer rule the largest R whose
    default capacity stays below 2^24.  2D Ising L=16 (a 32-byte row per replica, half a GB
    per spin buffer).  After two temperature steps, the third step's copy counts and ln Q
    equal the oracle's on the GPU's own pre-step energies, the counts sum to R_i, the
    ancestors follow from them, and sampled replicas swept by the oracle match bit for bit."""
    L, theta, seed, n = 16, 2, 5, 50
    rmax = (1 << 24) - 1
    R = rmax
    if rule == "nearest":
        while pa.default_capacity(R, rule) > rmax:
            R -= 1024
    betas = np.linspace(0.0, 0.8, n + 1)
    thetas = np.full(n, theta, np.uint32)
    g = pa.Population(2, L, R, betas, thetas, rule, seed)
    g.step(2)
    E_pre, words_pre = g.energies(), g.spins_words()
    g.step(1)
    i = 3
    obs = g.observables()
    ref = O.resample(E_pre, R, betas[i] - betas[i - 1], O.RESAMPLERS[rule], seed, i)
    assert ref["status"] == 0
    counts = g.counts()
    assert np.array_equal(counts, ref["counts"])
    assert obs["R_i"] == ref["R_new"] == int(counts.sum(dtype=np.int64))
    assert math.isclose(obs["lnQ"], ref["lnQ"], rel_tol=1e-12)
    anc = g.ancestors()
    assert np.array_equal(anc, np.repeat(np.arange(len(counts), dtype=np.uint32), counts))
    words, E = g.spins_words(), g.energies()
    J = O.ferro_couplings(2, L)
    N = L * L
    rng = np.random.default_rng(3)
    for d in list(rng.choice(obs["R_i"], 6, replace=False)) + [obs["R_i"] - 1]:
        parent = words_pre[anc[d]]
        bits = ((parent[:, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(-1)[:N]
        sig = (1 - 2 * bits.astype(np.int8)).astype(np.int8)
        s2, E2, _ = O.sweeps(2, L, J, sig, seed, i, int(d), theta, betas[i])
        assert np.array_equal(words[d], O.pack_spins(s2[None])[0]), (rule, d)
        assert E[d] == E2
    g.close()


def _curand_lib():
    out = os.path.join(tempfile.gettempdir(), f"philox_curand_ref_{os.getpid()}.so")
    if not os.path.exists(out):
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "philox_curand_ref.cu")],
                       check=True)
    lib = C.CDLL(out)
    lib.curand_philox_blocks.argtypes = [C.c_void_p] * 4 + [C.c_int]
    return lib


def test_philox_matches_curand():
    """Counter (c0, c1, c2, c3), key (k0, k1): cuRAND's curand_init(seed = k0 + 2^32 k1,
    subsequence = c2 + 2^32 c3, offset = 4 (c0 + 2^32 c1)) then curand4."""
    lib = _curand_lib()
    rng = np.random.default_rng(11)
    n = 400
    k = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64)
    c = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64)
    c[:, 1] &= np.uint64((1 << 30) - 1)   # the offset is 64-bit: 4 (c0 + 2^32 c1) < 2^64
    c[:50, 1] = 0
    seed = (k[:, 0] | (k[:, 1] << np.uint64(32))).astype(np.uint64)
    sub = (c[:, 2] | (c[:, 3] << np.uint64(32))).astype(np.uint64)
    off = ((c[:, 0] | (c[:, 1] << np.uint64(32))) * np.uint64(4)).astype(np.uint64)
    out = np.zeros((n, 4), np.uint32)
    assert lib.curand_philox_blocks(seed.ctypes.data, sub.ctypes.data, off.ctypes.data,
                                    out.ctypes.data, n) == 0
    for j in range(n):
        ref = O.philox([int(v) for v in c[j]], [int(k[j, 0]), int(k[j, 1])])
        assert np.array_equal(out[j], ref), j


@pytest.mark.parametrize("rule", ["systematic", "nearest"])
def test_free_energy_L16_reaches_kaufman(rule):
    """2D Ising L=16, beta 0 -> 1 in 100 steps, theta=10, R=100000: |f - f_exact| < 1e-4
    per spin at every step."""
    L, R, n = 16, 100000, 100
    betas = np.linspace(0.0, 1.0, n + 1)
    g = pa.Population(2, L, R, betas, np.full(n, 10, np.uint32), rule, 1)
    g.step(n)
    kf = _kaufman(L)
    worst = 0.0
    for row in g.trace():
        b = round(float(row["beta"]), 6)
        est = L * L * math.log(2) + row["sum_lnQ"]
        worst = max(worst, abs(est - kf[b]) / (L * L))
    assert worst < 1e-4
    g.close()


def test_free_energy_L64_all_rules():
    """The benchmark workload (L=64, R=100000, 200 steps to beta=1, theta=10): the
    estimator at beta_f is within 1e-4 per spin of Kaufman's exact value for every rule."""
    L, R, n = 64, 100000, 200
    betas = np.linspace(0.0, 1.0, n + 1)
    kf = _kaufman(L)
    for rule in RULES:
        g = pa.Population(2, L, R, betas, np.full(n, 10, np.uint32), rule, 7)
        g.step(n)
        mbf, f = g.free_energy()
        err = abs(mbf - kf[1.0]) / (L * L)
        assert err < 1e-4, (rule, err)
        g.close()
