"""Autotuner for the launch configuration of the sweep kernel.

The sweep kernel runs one CTA per 32 replicas; how many threads share a CTA
(64-512) trades per-CTA parallelism against the number of CTAs resident per
SM and the rounding of the grid into waves, which depends on the lattice and
on the population size.  The grouped 3D kernel has a fixed CTA size and holds
several replica groups per CTA; the tuner picks between that count and twice
it.  The tuner times each candidate on a throw-away run of
the same shape (same lattice, couplings kind, R and theta; results never
depend on the choice) and remembers the fastest per device and shape, in
memory and in a small JSON cache file.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import pa

CANDIDATES = (64, 128, 256, 384, 512)
_CACHE = {}
_CACHE_FILE = os.path.join(os.path.expanduser("~"), ".cache", "pa_gb300_tune.json")


def _key(dim, L, R, ea, theta):
    try:
        import torch
        dev = torch.cuda.get_device_name()
    except Exception:
        dev = "cuda"
    return f"{dev}|d{dim}|L{L}|R{R}|ea{int(ea)}|theta{theta}"


def _load():
    if _CACHE:
        return
    try:
        with open(_CACHE_FILE) as fh:
            _CACHE.update(json.load(fh))
    except Exception:
        pass


def _save():
    try:
        os.makedirs(os.path.dirname(_CACHE_FILE), exist_ok=True)
        with open(_CACHE_FILE, "w") as fh:
            json.dump(_CACHE, fh)
    except Exception:
        pass


def best_sweep_threads(dim, L, R, couplings=("ferro",), theta=10, candidates=CANDIDATES,
                       rounds=2, use_cache=True, stream=None):
    """Threads per CTA of the fastest sweep for this shape (timed on the current device)."""
    return best_sweep_threads_batch([{"dim": dim, "L": L, "R": R, "couplings": couplings}],
                                    theta=theta, candidates=candidates, rounds=rounds,
                                    use_cache=use_cache, stream=stream)


def _batch_key(specs, theta):
    try:
        import torch
        dev = torch.cuda.get_device_name()
    except Exception:
        dev = "cuda"
    if len(specs) == 1:
        s = specs[0]
        ea = s.get("couplings", ("ferro",))[0] != "ferro"
        return _key(s["dim"], s["L"], s["R"], ea, theta)
    shape = sorted((s["L"], s["R"], int(s.get("couplings", ("ferro",))[0] != "ferro"))
                   for s in specs)
    desc = hashlib.sha256(repr(shape).encode()).hexdigest()[:16]
    return f"{dev}|batch|d{specs[0]['dim']}|M{len(specs)}|{desc}|theta{theta}"


def best_sweep_threads_batch(specs, theta=10, candidates=CANDIDATES, rounds=2, use_cache=True,
                             stream=None):
    """Threads per CTA of the fastest sweep for a batch of runs (pa.Batch specs): every
    candidate is timed on a throw-away batch of the same runs (results never depend on the
    choice); the fastest is remembered per device and shape."""
    key = _batch_key(specs, theta)
    if use_cache:
        _load()
        if key in _CACHE:
            return int(_CACHE[key])
    n = rounds * len(candidates) + 1
    betas = np.linspace(0.0, 0.5, n + 1)
    thetas = np.full(n, theta, np.uint32)
    run = pa.Batch([dict(s) for s in specs], betas, thetas, "systematic", 12345, stream=stream,
                   graph=False)
    run.step(1)  # first launch of each kernel outside the timings
    best = {}
    pa.pa_enable_timing(run.ctx, True)
    for _ in range(rounds):
        for t in candidates:
            pa.pa_set_sweep_threads(run.ctx, t)
            run.step(1)
            ms, cnt, upd = pa.pa_sweep_timing(run.ctx)
            rate = upd / max(ms, 1e-9)
            best[t] = max(best.get(t, 0.0), rate)
    run.close()
    choice = max(best, key=best.get)
    _CACHE[key] = int(choice)
    if use_cache:
        _save()
    return int(choice)


def best_sweep_groups_batch(specs, theta=10, rounds=2, use_cache=True, stream=None):
    """Group multiple (1 or 2) of the fastest grouped 3D sweep for a batch of runs: 1 when
    the runs do not use the grouped kernel, else both are timed on a throw-away batch of
    the same runs (results never depend on the choice) and the faster is remembered."""
    if any(s["dim"] != 3 for s in specs):
        return 1
    key = _batch_key(specs, theta) + "|groups"
    if use_cache:
        _load()
        if key in _CACHE:
            return int(_CACHE[key])
    n = 2 * rounds + 1
    betas = np.linspace(0.0, 0.5, n + 1)
    thetas = np.full(n, theta, np.uint32)
    run = pa.Batch([dict(s) for s in specs], betas, thetas, "systematic", 12345, stream=stream,
                   graph=False)
    choice = 1
    try:
        pa.pa_set_sweep_groups(run.ctx, 2)
    except pa.PAError:
        run.close()  # the runs take the general kernel
    else:
        run.step(1)  # first launch of each kernel outside the timings
        best = {}
        pa.pa_enable_timing(run.ctx, True)
        for _ in range(rounds):
            for g in (1, 2):
                pa.pa_set_sweep_groups(run.ctx, g)
                run.step(1)
                ms, cnt, upd = pa.pa_sweep_timing(run.ctx)
                best[g] = max(best.get(g, 0.0), upd / max(ms, 1e-9))
        run.close()
        choice = max(best, key=best.get)
    _CACHE[key] = int(choice)
    if use_cache:
        _save()
    return int(choice)
