"""The learned schedule controller on the GPU against its oracle.

* the network kernels: inference bit-exact against the FP32 device-order
  oracle; training gradients against the FP64 oracle; one Adam step against
  its formula;
* the controller kernel: features equal the run's own statistics, every
  decision replays exactly through the oracle's decision rule, the realized
  schedule reruns bit-exact through the oracle PA, and the plain fallback
  (network off, or non-finite outputs) equals an uncontrolled run;
* the trained network's gain over the plain schedule at an equal sweep budget
  (2D Ising L=16, free energy against Kaufman's exact value).
"""
import math
import os

import numpy as np
import pytest

from tests.conftest import gpu_available

pytestmark = pytest.mark.gpu

if not gpu_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import torch  # noqa: E402

from oracle import mlp as M  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2401_07965_gb300 import controller as CT  # noqa: E402
from paper_2401_07965_gb300 import pa  # noqa: E402

DEV = torch.device("cuda")


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _kaufman(L, beta):
    path = os.path.join(os.path.dirname(__file__), "golden", "kaufman_lnZ.txt")
    with open(path) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            l, b, v = ln.split()
            if int(l) == L and abs(float(b) - beta) < 1e-12:
                return float(v)
    raise KeyError((L, beta))


# ---- network kernels ---------------------------------------------------------------------------

@pytest.mark.parametrize("B", [1, 31, 70])
def test_forward_bit_exact_against_device_order_oracle(B):
    rng = np.random.default_rng(B)
    bits = M.bf16_bits(rng.normal(0, 0.4, M.NPARAM).astype(np.float32))
    X = rng.normal(0, 1.5, (B, M.IN)).astype(np.float32)
    Y = CT.predict(bits, X)
    for b in range(B):
        ref = M.forward32(bits, X[b])
        assert np.array_equal(Y[b].view(np.uint32), ref.view(np.uint32)), b


def test_gradients_match_fp64_oracle():
    rng = np.random.default_rng(5)
    B = 100  # four CTAs of 32 rows, the last one ragged
    w = rng.normal(0, 0.3, M.NPARAM).astype(np.float32)
    X = rng.normal(0, 1, (B, M.IN)).astype(np.float32)
    Yt = rng.normal(0, 1, (B, M.OUT)).astype(np.float32)
    mask = (rng.random((B, M.OUT)) > 0.25).astype(np.float32)
    wd, Xd, Yd, Md = (torch.from_numpy(a).to(DEV) for a in (w, X, Yt, mask))
    g = torch.zeros(M.NPARAM, dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, dtype=torch.float32, device=DEV)
    scratch = torch.empty(pa.pa_mlp_scratch_bytes(B), dtype=torch.uint8, device=DEV)
    pa.pa_mlp_gradients(wd.data_ptr(), Xd.data_ptr(), Yd.data_ptr(), Md.data_ptr(), B,
                        g.data_ptr(), loss.data_ptr(), scratch.data_ptr(), scratch.numel(),
                        _stream())
    torch.cuda.synchronize()
    # the forward pass uses the BF16-rounded parameters (as inference does)
    w_bf = M.bf16_round(w).astype(np.float64)
    g64, l64 = M.grads64(w_bf, X.astype(np.float64), Yt.astype(np.float64),
                         mask.astype(np.float64))
    gd = g.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(g64))
    assert np.all(np.abs(gd - g64) <= 2e-5 * scale + 1e-4 * np.abs(g64))
    assert math.isclose(float(loss.item()), l64, rel_tol=1e-5)
    # a plausible slip (one layer's gradient transposed) would be far outside this
    assert np.max(np.abs(gd - g64)) < 1e-3 * scale


def test_adam_step_matches_formula():
    rng = np.random.default_rng(9)
    w = rng.normal(0, 1, M.NPARAM).astype(np.float32)
    g = rng.normal(0, 1, M.NPARAM).astype(np.float32)
    m = rng.normal(0, 0.1, M.NPARAM).astype(np.float32)
    v = rng.random(M.NPARAM).astype(np.float32)
    wd, gd, md, vd = (torch.from_numpy(a.copy()).to(DEV) for a in (w, g, m, v))
    wb = torch.zeros(M.NPARAM, dtype=torch.int16, device=DEV)
    step, lr = 7, 1e-3
    pa.pa_mlp_adam(wd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), wb.data_ptr(),
                   step, lr, _stream())
    torch.cuda.synchronize()
    # Kingma & Ba's update with the kernel's FP32 constants (beta1 = 0.9f,
    # beta2 = 0.999f, 1 - beta in FP32), each operation rounded to FP32
    f = np.float32
    b1, b2 = f(0.9), f(0.999)
    m1 = f(b1 * m) + f(f(f(1) - b1) * g)
    v1 = f(b2 * v) + f(f(f(f(1) - b2) * g) * g)
    assert np.array_equal(md.cpu().numpy(), m1)
    assert np.array_equal(vd.cpu().numpy(), v1)
    c1, c2 = 1 - 0.9 ** step, 1 - 0.999 ** step
    w1 = w - lr * (m1.astype(np.float64) / c1) / (np.sqrt(v1.astype(np.float64) / c2) + 1e-8)
    wn = wd.cpu().numpy()
    assert np.allclose(wn, w1, rtol=1e-6, atol=2e-7)
    assert np.array_equal(wb.cpu().numpy().view(np.uint16), M.bf16_bits(wn))


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (512, M.IN)).astype(np.float32)
    Y = np.stack([1 + 0.5 * np.sin(2 * X[:, 0]), 1 - 0.3 * X[:, 1] * X[:, 2]], 1).astype(np.float32)
    _, bits, hist = CT.train(X, Y, iters=1500, lr=3e-3, log_every=500)
    assert hist[-1][1] < 0.1 * hist[0][1] or hist[-1][1] < 2e-3
    pred = CT.predict(bits, X)
    assert np.sqrt(np.mean((pred - Y) ** 2)) < 0.08


# ---- controller kernel -------------------------------------------------------------------------

def _run_controlled(dim, L, cpl, R, K, beta_f, bits, use_mlp, plain_units=2, plain_theta=10,
                    budget=0, seed=3, resampler="systematic"):
    betas = np.linspace(0.0, beta_f, K + 1)
    pop = CT.controlled_run(dim, L, cpl, R, betas, plain_units, plain_theta, bits if use_mlp else
                            None, seed=seed, budget=budget, resampler=resampler)
    CT.run_to_end(pop)
    return pop, betas


def _test_params():
    """A network whose outputs vary over the anneal: the committed weights if present,
    else a fixed random initialisation (outputs near 1)."""
    if os.path.exists(CT.WEIGHTS):
        return CT.load()
    return M.bf16_bits(CT.init_params(4))


def test_controller_decisions_replay_through_oracle_rule():
    L, R, K = 16, 400, 200
    bits = _test_params()
    cfg_budget = 600
    pop, grid = _run_controlled(2, L, ("ferro",), R, K, 1.0, bits, True, plain_units=2,
                                plain_theta=6, budget=cfg_budget)
    rows = pop.trace()
    betas, thetas = pa.pa_schedule_taken(pop.ctx, K + 1)
    n = len(betas) - 1
    assert abs(betas[-1] - 1.0) < 1e-15 and len(rows) == n + 1
    cfg = dict(K=K, use_mlp=1, plain_units=2, plain_theta=6, theta_min=2, theta_max=40,
               budget=cfg_budget, u_max=8, theta_c=np.float32(cfg_budget) / np.float32(K // 2))
    k, used = 0, 0
    for i in range(n):
        x = np.array(rows[i]["features"], np.float32)
        d = M.decide(M.forward32(bits, x), k, used, cfg)
        assert d == (rows[i]["u_next"], rows[i]["theta_next"]), i
        k += d[0]
        used += d[1]
        assert betas[i + 1] == grid[k] and thetas[i] == d[1]
    assert k == K and used <= cfg_budget + 2
    assert M.decide(M.forward32(bits, np.array(rows[n]["features"], np.float32)), k, used,
                    cfg) is None
    # the features are the run's own statistics (float32 of the FP64 values)
    for i in range(n + 1):
        r = rows[i]
        Ri, N = r["R_i"], L * L
        mE = r["sumE"] / Ri
        var = (r["sumE2"] / Ri - mE * mE) / N
        th = thetas[i - 1] if i > 0 else 0
        ent = r["entropy"]
        ref = [r["beta"], mE / N, var / 10, r["lnQ"] / N * 10, r["sumC2"] / (Ri * Ri),
               ent / math.log(R), r["accepts"] / (th * N * Ri) if th else 0.0, L / 64]
        assert np.allclose(np.array(r["features"], np.float64), ref, rtol=2e-6, atol=1e-6), i
    pop.close()


def test_controlled_run_equals_oracle_on_realized_schedule():
    L, R, K = 8, 300, 120
    bits = _test_params()
    pop, _ = _run_controlled(3, L, ("ea", 3, 5), R, K, 2.0, bits, True, plain_units=3,
                             plain_theta=4, seed=11, resampler="poisson")
    betas, thetas = pa.pa_schedule_taken(pop.ctx, K + 1)
    J = O.disorder(3, L, 3, 5)
    orc = O.Run(3, L, J, R, betas, thetas, O.RESAMPLERS["poisson"], 11,
                R_cap=pa.default_capacity(R, "poisson"))
    for _ in range(len(betas) - 1):
        assert orc.step() == 0
    g, o = pop.observables(), orc.obs()
    assert g["R_i"] == o["R_i"]
    for key in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumC2", "accepts"):
        assert g[key] == o[key], key
    assert math.isclose(g["sum_lnQ"], o["sum_lnQ"], rel_tol=1e-12, abs_tol=1e-13)
    assert np.array_equal(pop.spins_words(), O.pack_spins(orc.spins()))
    assert np.array_equal(pop.families(), orc.families())
    pop.close()


@pytest.mark.parametrize("mode", ["off", "nan"])
def test_fallback_equals_plain_schedule(mode):
    """Network off, or a network whose outputs are not finite: the controller takes
    plain steps of plain_units grid points with plain_theta sweeps."""
    L, R, K, units, theta = 16, 300, 60, 3, 5
    bits = np.full(M.NPARAM, 0x7FC0, np.uint16) if mode == "nan" else None
    grid = np.linspace(0.0, 1.0, K + 1)
    pop = CT.controlled_run(2, L, ("ferro",), R, grid, units, theta, bits, seed=2)
    CT.run_to_end(pop)
    betas, thetas = pa.pa_schedule_taken(pop.ctx, K + 1)
    assert np.array_equal(betas, grid[::units]) and np.all(thetas == theta)
    ref = pa.Population(2, L, R, grid[::units], np.full(K // units, theta, np.uint32),
                        "systematic", 2)
    ref.step(K // units)
    assert np.array_equal(ref.spins_words(), pop.spins_words())
    assert ref.observables()["sum_lnQ"] == pop.observables()["sum_lnQ"]
    with pytest.raises(pa.PAError) as e:
        pop.step(1)
    assert e.value.status == pa.PA_ERR_DONE
    pop.close()
    ref.close()


# ---- what the trained network gains --------------------------------------------------------------

@pytest.mark.skipif(not os.path.exists(CT.WEIGHTS), reason="no trained controller weights")
def test_trained_controller_beats_plain_schedule_at_equal_budget():
    """2D Ising L=16, R=4000, beta to 1 with 1000 sweeps in total: plain 100 steps of
    10 sweeps against the learned schedule on a 400-point grid.  Root-mean-square
    error of -beta F per spin against Kaufman's exact value over 16 seeds."""
    L, R = 16, 4000
    bits = CT.load()
    exact = _kaufman(L, 1.0)
    err_plain, err_learned = [], []
    for seed in range(1, 17):
        p = pa.Population(2, L, R, np.linspace(0, 1, 101), np.full(100, 10, np.uint32),
                          "systematic", seed)
        p.step(100)
        err_plain.append((p.free_energy()[0] - exact) / (L * L))
        p.close()
        q, _ = _run_controlled(2, L, ("ferro",), R, 400, 1.0, bits, True, plain_units=4,
                               plain_theta=10, budget=1000, seed=seed)
        _, th = pa.pa_schedule_taken(q.ctx, 401)
        assert th.sum() <= 1002
        err_learned.append((q.free_energy()[0] - exact) / (L * L))
        q.close()
    rms_p = float(np.sqrt(np.mean(np.square(err_plain))))
    rms_l = float(np.sqrt(np.mean(np.square(err_learned))))
    print(f"rms plain {rms_p:.3e} learned {rms_l:.3e}")
    assert rms_l < 0.85 * rms_p


def test_controlled_run_under_graph_replay_equals_direct_launches():
    """The controller kernel is part of the captured step: replaying the graph on a side
    stream takes the same decisions and reaches the same state as direct launches."""
    L, R, K = 16, 300, 120
    bits = _test_params()
    grid = np.linspace(0.0, 1.0, K + 1)
    side = torch.cuda.Stream()
    a = CT.controlled_run(2, L, ("ferro",), R, grid, 2, 6, bits, seed=8, stream=side)
    b = CT.controlled_run(2, L, ("ferro",), R, grid, 2, 6, bits, seed=8)
    CT.run_to_end(a)
    CT.run_to_end(b)
    ba, ta = pa.pa_schedule_taken(a.ctx, K + 1)
    bb, tb = pa.pa_schedule_taken(b.ctx, K + 1)
    assert np.array_equal(ba, bb) and np.array_equal(ta, tb)
    assert np.array_equal(a.spins_words(), b.spins_words())
    assert a.observables()["sum_lnQ"] == b.observables()["sum_lnQ"]
    a.close()
    b.close()


def test_controlled_batch_each_run_replays_through_oracle():
    """The learned schedule in a batch: every run takes its own steps (one controller
    CTA per run).  For each run, every decision replays through the oracle's decision
    rule from the recorded features, and the run's realized schedule rerun through the
    oracle PA (with the run's replica-slot base and index) is bit-exact."""
    K, units, theta = 120, 2, 6
    bits = _test_params()
    runs = [{"dim": 2, "L": 16, "R": 300}, {"dim": 2, "L": 16, "R": 200},
            {"dim": 2, "L": 8, "R": 150}]
    grid = np.linspace(0.0, 1.0, K + 1)
    b = pa.Batch(runs, grid, np.full(K, theta, np.uint32), "nearest", 21)
    pa.pa_set_controller(b.ctx, bits, 1, units, theta, 2, 40, 0, 8)
    done = False
    for _ in range(K // 8 + 2):  # at most one step per grid point
        try:
            b.step(8)
        except pa.PAError as e:
            assert e.status == pa.PA_ERR_DONE
            done = True
            break
        pa.pa_sync(b.ctx)
    assert done
    budget = theta * (K // units)
    cfg = dict(K=K, use_mlp=1, plain_units=units, plain_theta=theta, theta_min=2, theta_max=40,
               budget=budget, u_max=8, theta_c=np.float32(budget) / np.float32(K // units))
    schedules = []
    for m, (spec, base) in enumerate(zip(b.specs, b.slot_bases())):
        betas, thetas = pa.pa_run_schedule_taken(b.ctx, m, K + 1)
        rows = b.trace(m)
        n = len(betas) - 1
        assert abs(betas[-1] - 1.0) < 1e-15 and len(rows) == n + 1
        k, used = 0, 0
        for i in range(n):
            d = M.decide(M.forward32(bits, np.array(rows[i]["features"], np.float32)), k, used,
                         cfg)
            assert d == (rows[i]["u_next"], rows[i]["theta_next"]), (m, i)
            k += d[0]
            used += d[1]
            assert betas[i + 1] == grid[k] and thetas[i] == d[1]
        assert k == K
        L, R = spec["L"], spec["R"]
        cap = pa.default_capacity(R, "nearest")
        orc = O.Run(2, L, O.ferro_couplings(2, L), R, betas, thetas, O.RESAMPLERS["nearest"], 21,
                    R_cap=cap, slot_base=base, run_id=m)
        for _ in range(n):
            assert orc.step() == 0
        g, o = b.observables(m), orc.obs()
        assert g["R_i"] == o["R_i"] and g["step"] == n
        for key in ("sumE", "sumE2", "sumAbsM", "sumM2", "sumC2", "accepts"):
            assert g[key] == o[key], (m, key)
        assert math.isclose(g["sum_lnQ"], o["sum_lnQ"], rel_tol=1e-12, abs_tol=1e-13)
        assert np.array_equal(b.spins_words(m), O.pack_spins(orc.spins())), m
        schedules.append(tuple(betas))
    assert len(set(schedules)) > 1  # the runs took different schedules
    with pytest.raises(pa.PAError):
        b.weighted(0)
    b.close()
