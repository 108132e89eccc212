"""Host logic of the launch-shape autotuner, with the library calls replaced by fakes
(no GPU): the fastest candidate wins, the choice is cached per shape and device,
the group-multiple tuner leaves non-3D batches and contexts without the grouped
kernel at 1, and the two tuners keep separate cache entries."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2401_07965_gb300 import tune  # noqa: E402


class _Fake:
    """Stands in for pa.Batch and the timing/setting calls; rates[c] is the sweep rate
    the fake reports for launch setting c."""

    def __init__(self, rates, groups_ok=True):
        self.rates, self.groups_ok = rates, groups_ok
        self.batches = 0
        self.setting = None
        self.stepped = 0

    def install(self, mp):
        fake = self

        class Batch:
            def __init__(self, specs, betas, thetas, rule, seed, stream=None, graph=True):
                fake.batches += 1
                self.ctx = object()

            def step(self, n):
                fake.stepped += n

            def close(self):
                pass

        def set_threads(ctx, t):
            fake.setting = t

        def set_groups(ctx, g):
            if not fake.groups_ok:
                raise tune.pa.PAError(1, "pa_set_sweep_groups")
            fake.setting = g

        def timing(ctx):
            r = fake.rates.get(fake.setting, 1.0)
            return 1.0, 1, r * 1.0  # ms, launches, updates

        mp.setattr(tune.pa, "Batch", Batch)
        mp.setattr(tune.pa, "pa_set_sweep_threads", set_threads)
        mp.setattr(tune.pa, "pa_set_sweep_groups", set_groups)
        mp.setattr(tune.pa, "pa_sweep_timing", timing)
        mp.setattr(tune.pa, "pa_enable_timing", lambda ctx, on: None)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "_CACHE_FILE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(tune, "_CACHE", {})
    return tmp_path / "tune.json"


SPEC2 = [{"dim": 2, "L": 64, "R": 100000, "couplings": ("ferro",)}]
SPEC3 = [{"dim": 3, "L": 8, "R": 5000, "couplings": ("ea", 3, 1)},
         {"dim": 3, "L": 6, "R": 7000, "couplings": ("ea", 3, 2)}]


def test_fastest_threads_win_and_are_cached(cache, monkeypatch):
    f = _Fake({64: 1.0, 128: 3.0, 256: 2.0, 384: 0.5, 512: 1.5})
    f.install(monkeypatch)
    assert tune.best_sweep_threads_batch(SPEC2) == 128
    assert f.batches == 1 and cache.exists()
    # cached: no second throw-away batch, also after the in-memory cache is dropped
    assert tune.best_sweep_threads_batch(SPEC2) == 128
    monkeypatch.setattr(tune, "_CACHE", {})
    assert tune.best_sweep_threads_batch(SPEC2) == 128
    assert f.batches == 1
    # another shape is tuned again
    other = [dict(SPEC2[0], R=50000)]
    f.rates = {256: 9.0}
    assert tune.best_sweep_threads_batch(other) == 256
    assert f.batches == 2


def test_batch_key_ignores_run_order_but_not_sizes():
    a = tune._batch_key(SPEC3, 10)
    b = tune._batch_key(list(reversed(SPEC3)), 10)
    c = tune._batch_key([SPEC3[0], dict(SPEC3[1], R=7001)], 10)
    assert a == b and a != c
    assert tune._batch_key(SPEC3, 10) != tune._batch_key(SPEC3, 5)


def test_group_multiple(cache, monkeypatch):
    f = _Fake({1: 2.0, 2: 3.0})
    f.install(monkeypatch)
    assert tune.best_sweep_groups_batch(SPEC2) == 1       # not a 3D batch: no trial
    assert f.batches == 0
    assert tune.best_sweep_groups_batch(SPEC3) == 2
    assert f.batches == 1
    f.rates = {1: 5.0, 2: 3.0}
    assert tune.best_sweep_groups_batch(SPEC3) == 2       # cached
    assert tune.best_sweep_groups_batch(SPEC3, use_cache=False) == 1
    # the threads tuner of the same shape has its own entry
    f.rates = {512: 7.0}
    assert tune.best_sweep_threads_batch(SPEC3) == 512


def test_group_multiple_without_grouped_kernel(cache, monkeypatch):
    f = _Fake({1: 1.0, 2: 9.0}, groups_ok=False)
    f.install(monkeypatch)
    assert tune.best_sweep_groups_batch(SPEC3, use_cache=False) == 1
