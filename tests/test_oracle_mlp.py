"""Pins of the controller network's reference (oracle/mlp.py)."""
import numpy as np

from oracle import mlp


def _params(seed):
    rng = np.random.default_rng(seed)
    flat = rng.normal(0, 0.3, mlp.NPARAM).astype(np.float32)
    return mlp.bf16_round(flat).astype(np.float64)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    X = rng.normal(0, 1, (16, mlp.IN))
    Yt = rng.normal(0, 1, (16, mlp.OUT))
    mask = (rng.random((16, mlp.OUT)) > 0.2).astype(np.float64)
    g, loss = mlp.grads64(p, X, Yt, mask)
    h = 1e-6
    for idx in rng.choice(mlp.NPARAM, 60, replace=False):
        e = np.zeros(mlp.NPARAM)
        e[idx] = h
        lp = mlp.grads64(p + e, X, Yt, mask)[1]
        lm = mlp.grads64(p - e, X, Yt, mask)[1]
        assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-6 + 1e-5 * abs(g[idx])


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.00390625, 1.005859375, -2.5e-3, 3.0e38, 0.0], np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0          # tie to even
    assert r[2] == np.float32(1.0078125)        # above the tie
    assert abs(r[3] - x[3]) <= abs(x[3]) * 2 ** -8
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)


def test_fp32_forward_is_close_to_fp64():
    p = _params(3)
    bits = mlp.bf16_bits(p.astype(np.float32))
    x = np.linspace(-1, 1, mlp.IN).astype(np.float32)
    y32 = mlp.forward32(bits, x)
    y64, _ = mlp.forward64(mlp.bf16_to_f32(bits).astype(np.float64), x[None].astype(np.float64))
    assert np.allclose(y32, y64[0], rtol=1e-5, atol=1e-5)


def test_decision_rule_respects_budget_and_grid():
    cfg = dict(K=600, use_mlp=1, plain_units=2, plain_theta=10, theta_min=2, theta_max=40,
               budget=3000, u_max=8, theta_c=np.float32(3000 / 300))
    k, used, steps = 0, 0, 0
    rng = np.random.default_rng(0)
    while True:
        d = mlp.decide(np.array([rng.uniform(0.2, 5), rng.uniform(0.3, 3)], np.float32), k,
                       used, cfg)
        if d is None:
            break
        u, th = d
        assert 1 <= u <= 8 and 2 <= th <= 40
        k += u
        used += th
        steps += 1
    assert k == 600 and used <= 3000 + 2
    # plain fallback on non-finite outputs
    assert mlp.decide(np.array([np.nan, 1.0], np.float32), 0, 0, cfg) == (2, 10)
