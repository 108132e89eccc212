"""Pins of the oracle's random numbers and of its own exp.

Philox4x32-10 has no printed test vectors in the paper and none is typed in
here; it is pinned by its statistical properties on the CPU and, on the GPU,
against an independent library implementation (cuRAND's Philox generator).
"""
import math

import numpy as np
import pytest


def _outputs(O, n, key=(1, 0), c1=0):
    out = np.zeros((n, 4), np.uint32)
    for i in range(n):
        out[i] = O.philox([i, c1, 7, 3], key)
    return out


def test_philox_uniform_bytes(oracle):
    x = _outputs(oracle, 20000).view(np.uint8).ravel()
    counts = np.bincount(x, minlength=256)
    exp = len(x) / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 255 degrees of freedom: mean 255, sd ~22.6
    assert chi2 < 255 + 6 * 22.6


def test_philox_bit_balance_and_avalanche(oracle):
    x = _outputs(oracle, 4000)
    bits = np.unpackbits(x.view(np.uint8)).reshape(-1, 128)
    p = bits.mean(axis=0)
    assert np.all(np.abs(p - 0.5) < 0.06)
    # flipping any single counter or key bit changes about half the output bits
    base = oracle.philox([12345, 678, 9, 10], [0xDEADBEEF, 0x1234])
    flips = []
    for word in range(4):
        for b in range(32):
            c = [12345, 678, 9, 10]
            c[word] ^= 1 << b
            y = oracle.philox(c, [0xDEADBEEF, 0x1234])
            flips.append(sum(bin(int(u) ^ int(v)).count("1") for u, v in zip(base, y)))
    for b in range(64):
        k = [0xDEADBEEF, 0x1234]
        k[b // 32] ^= 1 << (b % 32)
        y = oracle.philox([12345, 678, 9, 10], k)
        flips.append(sum(bin(int(u) ^ int(v)).count("1") for u, v in zip(base, y)))
    flips = np.array(flips)
    assert flips.min() > 35 and flips.max() < 93
    assert abs(flips.mean() - 64) < 3


def test_philox_is_a_function_of_key_and_counter(oracle):
    a = oracle.philox([1, 2, 3, 4], [5, 6])
    assert np.array_equal(a, oracle.philox([1, 2, 3, 4], [5, 6]))
    assert not np.array_equal(a, oracle.philox([1, 2, 3, 4], [5, 7]))
    assert not np.array_equal(a, oracle.philox([1, 2, 3, 5], [5, 6]))


def test_philox_serial_correlation(oracle):
    u = _outputs(oracle, 20000).ravel().astype(np.float64) / 2 ** 32
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) < 5 / math.sqrt(len(u))
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(u))


def test_own_exp_accuracy(oracle):
    xs = np.concatenate([np.linspace(-16, 0, 20001), -np.logspace(-12, 1.2, 2000)])
    worst = 0.0
    for x in xs:
        got, ref = oracle.exp(float(x)), math.exp(float(x))
        worst = max(worst, abs(got - ref) / ref)
    assert worst < 4e-16
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-math.log(2)) == pytest.approx(0.5, rel=2e-16)


def _u_full(O, seed, slot, step, sweep, colour, site):
    """u assembled bit by bit: bit 31-p is bit (slot & 31) of plane word p."""
    u = 0
    for p in range(32):
        x = O.philox([slot >> 5, (sweep << 4) | (colour << 3) | (p >> 2), step, site],
                     [seed & 0xFFFFFFFF, seed >> 32])
        u |= ((int(x[p & 3]) >> (slot & 31)) & 1) << (31 - p)
    return u


def test_metropolis_uniform_digit_comparison_equals_full_comparison(oracle):
    """The oracle decides u < thr four bits at a time from the top; that must equal the
    comparison of the fully assembled 32-bit u, including thresholds close to u."""
    rng = np.random.default_rng(4)
    for _ in range(150):
        seed = int(rng.integers(0, 2 ** 63))
        slot, step = int(rng.integers(0, 5000)), int(rng.integers(1, 300))
        sweep, colour, site = int(rng.integers(0, 10)), int(rng.integers(0, 2)), int(
            rng.integers(0, 4096))
        u = _u_full(oracle, seed, slot, step, sweep, colour, site)
        for thr in (int(rng.integers(0, 2 ** 32)), u, u + 1, max(u - 1, 0), u ^ 1, u ^ 0x100,
                    0, 0xFFFFFFFF):
            thr &= 0xFFFFFFFF
            assert oracle.u_less(seed, slot, step, sweep, colour, site, thr) == (u < thr)


def test_metropolis_uniform_acceptance_rate(oracle):
    """P(u < thr) = thr / 2^32 for the bit-plane uniforms."""
    thr = int(0.3 * 2 ** 32)
    hits = sum(oracle.u_less(7, slot, 3, 0, 0, site, thr)
               for slot in range(0, 64) for site in range(0, 400, 2))
    n = 64 * 200
    assert abs(hits / n - 0.3) < 5 * math.sqrt(0.21 / n)
