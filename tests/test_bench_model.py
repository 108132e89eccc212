"""Host logic of bench.py (no GPU): the sweep roofline model and the clock summary.

The model counts, per site word (one site of 32 replicas), the integer work of the
bit-plane Metropolis test with an ideal stop at the first deciding plane block.
Its pieces are checked against what they stand for: E_B against a direct
simulation of the plane-by-plane decision, the zero-class boundaries against
exp(-beta dE) = 2^-8, and the per-class savings against the counts they drop.
"""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_expected_blocks_match_a_simulation_of_the_decision():
    """E_B = expected number of 4-plane blocks until every one of 32 replicas has a
    uniform that differs from its threshold in some drawn plane."""
    rng = np.random.default_rng(5)
    trials = 200_000
    u = rng.integers(0, 2 ** 32, size=(trials, 32), dtype=np.uint64)
    t = rng.integers(0, 2 ** 32, size=(trials, 32), dtype=np.uint64)
    x = u ^ t
    # blocks needed by a replica: 1 + (leading zero bits of u ^ t) // 4, capped at 8
    lz = np.where(x == 0, 32, 31 - np.floor(np.log2(np.maximum(x, 1))).astype(np.int64))
    need = np.minimum(1 + lz // 4, 8).max(axis=1)
    assert abs(need.mean() - bench.E_BLOCKS) < 0.01
    assert abs(bench.E_BLOCKS - 2.0) < 0.01
    assert bench.HEAD_BLOCKS == pytest.approx(1.0 + (1.0 - (15.0 / 16.0) ** 32))


def test_full_model_counts():
    p2, p3 = bench.pipes_model(2), bench.pipes_model(3)
    assert p2["alu"][0] == pytest.approx(62.0, abs=0.05)
    assert p2["fma"][0] == pytest.approx(76.0, abs=0.05)
    assert p2["issue"][0] == pytest.approx(108.0, abs=0.05)
    assert p3["alu"][0] == pytest.approx(72.0, abs=0.05)
    assert p3["fma"][0] == pytest.approx(84.0, abs=0.05)
    assert p3["issue"][0] == pytest.approx(126.0, abs=0.05)
    # issue = every counted instruction once; wide products take two FMA cycles
    for d in (2, 3):
        for z in range(4 if d == 3 else 3):
            m = bench.pipes_model(d, z)
            imad = m["fma"][0] - 2 * bench.MULWIDE_PER_SITEWORD
            assert m["issue"][0] == pytest.approx(m["alu"][0] + bench.MULWIDE_PER_SITEWORD + imad)


@pytest.mark.parametrize("d", [2, 3])
def test_zero_class_boundaries(d):
    ln256 = math.log(256.0)
    ks = (2, 1) if d == 2 else (3, 2, 1)
    assert bench.zero_classes(d, 0.0) == 0
    for n, k in enumerate(ks):
        edge = ln256 / (4 * k)
        assert bench.zero_classes(d, edge * (1 - 1e-9)) == n
        assert bench.zero_classes(d, edge * (1 + 1e-9)) == n + 1
    assert bench.zero_classes(d, 50.0) == len(ks)


@pytest.mark.parametrize("d", [2, 3])
def test_each_zero_class_drops_its_multiply_adds(d):
    ncls = 2 if d == 2 else 3
    prev = None
    for z in range(ncls + 1):
        m = bench.pipes_model(d, z)
        if prev is not None:
            dropped = prev["fma"][0] - m["fma"][0]
            # one multiply-add per plane of blocks 0 and 1, weighted as in E_B
            assert dropped == pytest.approx(4 * bench.HEAD_BLOCKS)
            assert m["alu"][0] <= prev["alu"][0]
        prev = m
    # with every class zero the compare takes 4 logic operations for the 8 planes
    full, zero = bench.pipes_model(d, 0), bench.pipes_model(d, ncls)
    assert full["alu"][0] - zero["alu"][0] == pytest.approx(4 * 1.5 * bench.HEAD_BLOCKS)


def test_mean_over_steps_weights_steps_equally():
    betas = [0.1, 0.1, 0.1, 0.8]
    m, hist = bench.mean_pipes(2, betas)
    assert hist == {0: 3, 1: 1}
    a, b = bench.pipes_model(2, 0), bench.pipes_model(2, 1)
    for k in m:
        assert m[k][0] == pytest.approx((3 * a[k][0] + b[k][0]) / 4)


def test_clock_summary_reads_throttle_reasons():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unavailable"]
    c.lines = [
        "0, 2070, 2070, 850.10, 0x0000000000000000, Not Active, Not Active, Not Active, "
        "Not Active",
        "0, 1980, 2070, 1400.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, 2040, 2070, 1390.00, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
