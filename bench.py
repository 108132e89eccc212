#!/usr/bin/env python3
"""Benchmark of the population-annealing hot path on one GB300 (or N, one run per GPU).

Workload (the headline configuration): 2D Ising ferromagnet, L=64 periodic,
R=100000 replicas, beta from 0 to 1 in 200 equal steps, theta=10 Metropolis
sweeps per step, one run for each of the five copy-count rules (multinomial,
systematic, residual, Poisson, nearest-integer), Philox seed 7.  One benchmark
"step" is one temperature step of one run (reweighting, Q, copy counts, scan,
gather, theta sweeps, measurements); the default 1000 steps are the five runs
back to back.  Inputs are synthetic (the method draws its own initial state).

Printed: one JSON line on rank 0.  `value` is spin updates per ns over the
timed steps (device time, CUDA events on the library's stream, L2 flushed
between steps); `roofline` relates the sweep kernel's integer throughput to
the SM issue peak; `e2e` times the same runs through the C ABI from host
arrays to host results; `cpu_baseline` times the CPU oracle on a bounded
sample of the same workload.

--impl reference times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("spin updates/ns and PA steps/s at 1 GB300 vs roofline; "
          "time-to-1e-4 free-energy error")
UNIT = "spin updates/ns"
RULES = ["multinomial", "systematic", "residual", "poisson", "nearest"]
L, DIM, R, NSTEPS, THETA, SEED, BETA_F = 64, 2, 100_000, 200, 10, 7, 1.0
WORKLOAD = ("2D Ising ferromagnet L=64 periodic, R=100000, beta 0->1 in 200 steps, theta=10, "
            "multinomial/systematic/residual/Poisson/nearest-integer runs, seed 7")
# Roofline of the sweep kernel (integer pipes).  Per site word (one site of the
# 32 replicas of a CTA) the bit-plane Metropolis test needs, with an ideal
# per-site stop at the first deciding plane block, E_B Philox blocks, where
# E_B = sum_g P(some replica undecided after 4g planes) = sum_g 1-(1-16^-g)^32.
# Per block: 14 wide multiplies (rounds 4-10; rounds 1-3 are shared by the
# counter layout) and 17 logic operations (their 14 three-input XORs and 3 to
# combine the shared halves); per plane, for d = 2, the replicas' threshold bit
# word as c4 b4 + c8 b8 (the two classes' masks are disjoint, bits 0/1: one
# multiply and one multiply-add) and 2 logic operations (the borrow and the
# "equal so far" words).  Per site: 2 wide multiplies (rounds 2-3) and 12 logic
# operations (four neighbour XORs, the class masks, the flip).
# Pipes per SM and clock: the integer ALU pipe takes 64 lane-operations (ncu:
# sm__inst_executed_pipe_alu peak = 2 warp instructions per cycle), the
# multiply (FMA-heavy) pipe 64 lane-operations with a 32x32->64 product taking
# two of them (a probe measured 25-28 products per clock per SM), and the
# schedulers issue 4 warp instructions (128 lane-instructions).  The roofline is
# set by the most loaded of the three.
E_BLOCKS = sum(1.0 - (1.0 - 16.0 ** -g) ** 32 for g in range(8))
# weights of plane blocks 0 and 1 in E_B; the kernels draw these two for every site
HEAD_BLOCKS = 1.0 + (1.0 - (15.0 / 16.0) ** 32)
MULWIDE_PER_SITEWORD = 2 + E_BLOCKS * 14
ALU_LANES_PER_SM = 64
FMA_LANES_PER_SM = 64
ISSUE_LANES_PER_SM = 128


def zero_classes(d, beta):
    """Energy classes (dE = 4k, from the highest down) whose threshold exp(-beta dE)
    is below 2^-8, i.e. has eight zero top bits: their threshold terms vanish in plane
    blocks 0 and 1, which the kernels then leave out."""
    zc = 0
    for k in range(2 if d == 2 else 3, 0, -1):
        if math.exp(-4.0 * k * beta) >= 2.0 ** -8:
            break
        zc += 1
    return zc


def pipes_model(d, zc=0):
    """Per-site-word demand on the three integer resources (see the comment above).
    d = 3: six bonds, classes dE = 4, 8, 12: per site 22 logic operations (six
    neighbour XORs, the bit-sliced count of unsatisfied bonds, the class masks, the
    flip) and per plane one multiply and two multiply-adds for the threshold word.
    zc classes with eight zero top threshold bits need no multiply-add in blocks 0
    and 1; with none left (t = 0) the borrow is 0 and the equality word takes 4 logic
    operations for the 8 planes."""
    ncls = 2 if d == 2 else 3
    nc = ncls - zc
    tail = E_BLOCKS - HEAD_BLOCKS
    cmp_logic = 4 * (2.0 if nc > 0 else 0.5) * HEAD_BLOCKS + 4 * 2 * tail
    imad = 4 * nc * HEAD_BLOCKS + 4 * ncls * tail
    alu = (12 if d == 2 else 22) + E_BLOCKS * 17 + cmp_logic
    fma = 2 * MULWIDE_PER_SITEWORD + imad
    issue = alu + MULWIDE_PER_SITEWORD + imad
    return {"alu": (alu, ALU_LANES_PER_SM), "fma": (fma, FMA_LANES_PER_SM),
            "issue": (issue, ISSUE_LANES_PER_SM)}


def mean_pipes(d, betas):
    """pipes_model averaged over timed steps at inverse temperatures `betas` (equal
    work per step), and how many steps had each number of zero classes."""
    models = [pipes_model(d, zero_classes(d, b)) for b in betas]
    out = {k: (sum(m[k][0] for m in models) / len(models), models[0][k][1]) for k in models[0]}
    hist = {}
    for b in betas:
        z = zero_classes(d, b)
        hist[z] = hist.get(z, 0) + 1
    return out, hist


def roofline_record(pipes, rate, nsm, f_hz):
    """Binding pipe of the per-site-word demand `pipes` and the fraction reached at `rate`
    spin updates/ns."""
    bind = max(pipes, key=lambda k: pipes[k][0] / pipes[k][1])
    per_sw, lanes = pipes[bind]
    peak = nsm * lanes * f_hz / 1e12
    achieved = per_sw / 32.0 * rate * 1e9 / 1e12
    return {"bound": "alu", "binding_pipe": bind, "achieved": achieved, "peak": peak,
            "unit": "T lane-ops/s", "frac": achieved / peak,
            "roofline_updates_per_ns": peak * 1e3 * 32.0 / per_sw,
            "per_site_word": {k: v[0] for k, v in pipes.items()}}


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _sweep_traffic(kernel_src_hash):
    """DRAM bytes per sweep launch from a committed ncu capture of the current kernel source."""
    path = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("kernel_source_sha256") != kernel_src_hash:
        return None
    return d.get("dram_bytes_per_full_launch")


def _src_hash():
    h = hashlib.sha256()
    for f in ("pa_sweep2d.cu", "pa_sweep_common.cuh", "pa_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2401_07965_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


# ----------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(R_s, beta_i, rule="systematic", parallel=False):
    """Time the CPU oracle on one temperature step of the benchmark schedule at inverse
    temperature beta_i (theta=10 sweeps and the resampling into it) for a population of
    R_s replicas of the benchmark lattice.  The population reaches beta_i - 1/200 in one
    untimed step without sweeps.  parallel: the OpenMP build on all host cores.
    Returns (updates, seconds)."""
    from oracle import oracle as O
    O.build()
    db = BETA_F / NSTEPS
    betas = np.array([0.0, max(beta_i - db, db / 2), beta_i])
    thetas = np.array([0, THETA], np.uint32)
    run = O.Run(DIM, L, O.ferro_couplings(DIM, L), R_s, betas, thetas, O.RESAMPLERS[rule], SEED,
                R_cap=4 * R_s, parallel=parallel)
    assert run.step() == 0
    t0 = time.perf_counter()
    assert run.step() == 0
    sec = time.perf_counter() - t0
    return THETA * L * L * run.size, sec


def oracle_baseline(R_s, n_samples, parallel):
    """The oracle on n_samples temperature steps spread over the schedule (rules cycled);
    returns the cpu_baseline record."""
    upd, sec = 0, 0.0
    for k in range(n_samples):
        i = 1 + (k * NSTEPS) // n_samples + NSTEPS // (2 * n_samples)
        u, t = oracle_sample(R_s, BETA_F * i / NSTEPS, RULES[k % 5], parallel)
        upd += u
        sec += t
    cores = host_cores() if parallel else 1
    what = ("OpenMP build of the CPU oracle (replica loop of the sweeps on all %d host cores)"
            % cores if parallel else "CPU oracle, single thread")
    return {"value": upd / (sec * 1e9), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s, one int8 per spin: %d temperature steps spread over the schedule "
                      "(beta 0->1, rules cycled), each %d replicas of the L=64 lattice through "
                      "resampling + theta=10 sweeps; %.2e updates in %.1f s"
                      % (what, n_samples, R_s, upd, sec)}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    R_s = 1024
    cores = host_cores()
    for k in range(args.warmup):
        oracle_sample(R_s // 4, BETA_F * 0.5, RULES[k % 5], parallel=True)
    upd_tot, sec_tot = 0, 0.0
    for k in range(args.steps):
        i = 1 + (k * NSTEPS) // args.steps + NSTEPS // (2 * args.steps)
        u, s = oracle_sample(R_s, BETA_F * i / NSTEPS, RULES[k % 5], parallel=True)
        upd_tot += u
        sec_tot += s
    v = upd_tot / (sec_tot * 1e9)
    sample = (f"each step: the CPU oracle (OpenMP build, {cores} host cores) runs {R_s} "
              f"replicas of the L=64 lattice through one temperature step (resampling + "
              f"theta=10 sweeps) at a beta spread over the schedule, rules cycled over the five")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_replicas": R_s},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def combine_over_ranks(ms, units, device):
    """Whole-job figures of independent runs on several ranks: the maximum of the ranks'
    device times and the sum of their units (one all-reduce each; no data-path exchange)."""
    import torch
    import torch.distributed as dist
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    t_units = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_units, op=dist.ReduceOp.SUM)
    return float(t_ms[0]), float(t_units[0])


def rank_seed(rank):
    """Each rank runs its own population: the Philox key is offset by the rank."""
    return SEED + 1000 * rank


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------

def timed_positions(K):
    """Which of the benchmark's steps are timed.  The five runs (one per rule) take
    5 x 200 = 1000 temperature steps.  K >= 1000: the first K steps (the runs repeat).
    K < 1000: all 1000 steps run and K of them, spread evenly over the five rules and the
    whole beta schedule, are timed (step p_k = floor((k + 1/2) 1000 / K))."""
    total = NSTEPS * len(RULES)
    if K >= total:
        return K, list(range(K))
    return total, sorted({int((k + 0.5) * total / K) for k in range(K)})


def run_ours(args):
    import torch
    rank, world, local = _env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2401_07965_gb300 import pa

    betas = np.linspace(0.0, BETA_F, NSTEPS + 1)
    thetas = np.full(NSTEPS, THETA, np.uint32)
    seed = rank_seed(rank)
    stream = torch.cuda.current_stream(dev)

    # launch configuration of the sweep from the autotuner (timed on this GPU, cached)
    from paper_2401_07965_gb300 import tune
    threads = tune.best_sweep_threads(DIM, L, R, theta=THETA, stream=stream)

    # warm-up on a throw-away run of the same shape
    wu = pa.Population(DIM, L, R, betas, thetas, "systematic", seed + 99, stream=stream,
                       sweep_threads=threads)
    wu.step(max(args.warmup, 1))
    wu.observables()
    wu.close()

    n_run, timed = timed_positions(args.steps)
    timed_set = set(timed)
    K = len(timed)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    timed_steps = []          # (rule, step index within its run)
    launches = 0
    updates = 0.0
    sweep_ms, sweep_n, sweep_upd = 0.0, 0, 0.0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    pos, k = 0, 0
    with ClockSampler(local) as clk:
        r = 0
        while pos < n_run:
            rule = RULES[r % len(RULES)]
            n = min(NSTEPS, n_run - pos)
            p = pa.Population(DIM, L, R, betas, thetas, rule, seed, stream=stream,
                              sweep_threads=threads)
            pa.pa_enable_timing(p.ctx, True)     # creates the event pool outside the steps
            pa.pa_enable_timing(p.ctx, False)
            mine = []
            for i in range(1, n + 1):
                if pos in timed_set:
                    flush.fill_(k & 0xFF)          # L2 flush, outside the step's events
                    pa.pa_enable_timing(p.ctx, True)
                    l0 = pa.pa_launch_count(p.ctx)
                    ev[k][0].record(stream)
                    p.step(1)
                    ev[k][1].record(stream)
                    launches += pa.pa_launch_count(p.ctx) - l0
                    pa.pa_enable_timing(p.ctx, False)
                    mine.append(i)
                    timed_steps.append((rule, i))
                    k += 1
                else:
                    p.step(1)                       # untimed, replayed as a CUDA graph
                pos += 1
            tr = p.trace()
            updates += sum(THETA * L * L * tr[i]["R_i"] for i in mine)
            ms, cnt, u = pa.pa_sweep_timing(p.ctx)
            sweep_ms += ms
            sweep_n += cnt
            sweep_upd += u
            p.close()
            r += 1
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    # max over ranks of the device time; sum of the units
    if world > 1:
        total_ms, updates = combine_over_ranks(total_ms, updates, dev)
    value = updates / (total_ms * 1e6)
    del flush

    # end to end through the C ABI from host inputs to host results
    e2e = None if args.no_e2e else run_e2e(args, pa, stream, seed, dev, threads)
    # time to a free energy within 1e-4 per spin of Kaufman's value (L=64)
    acc = None if (args.no_accuracy or world > 1) else accuracy_l64(pa, dev)
    # the batched 3D spin-glass workload (192 runs), 20 steps spread over its schedule
    ea3d = None if (args.no_ea3d or world > 1) else ea3d_batch(pa, stream, 64, 20, 5,
                                                               timed_sweeps=True)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    clocks = clk.summary()
    f_hz = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    sweep_rate = sweep_upd / (sweep_ms * 1e6)  # updates / ns inside the sweep kernel
    # the model's demand averaged over the timed steps' temperatures
    pipes_t, zc_hist = mean_pipes(DIM, [betas[i] for _, i in timed_steps])
    binding = max(pipes_t, key=lambda k: pipes_t[k][0] / pipes_t[k][1])
    per_sw, lanes = pipes_t[binding]
    peak = nsm * lanes * f_hz / 1e12                       # T lane-operations / s
    achieved = per_sw / 32.0 * sweep_rate * 1e9 / 1e12
    traffic_full = _sweep_traffic(_src_hash())
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-ops/s",
            "frac": achieved / peak, "traffic": traffic_full,
            "kernel": "k_sweep2d<64,T,false> (gather + theta bit-plane Metropolis sweeps + "
                      "measure)",
            "binding_pipe": binding,
            "peak_source": f"{nsm} SMs x {lanes} lanes of the {binding} pipe x sm_max_mhz "
                           f"({peak_src} clocks); lanes per pipe from ncu's pipe peaks",
            "per_site_word": {k: v[0] for k, v in pipes_t.items()},
            "zero_class_steps": {str(z): c for z, c in sorted(zc_hist.items())},
            "pipe_fracs": {k: v[0] / 32.0 * sweep_rate * 1e9 / (nsm * v[1] * f_hz)
                           for k, v in pipes_t.items()},
            "sweep_updates_per_ns": sweep_rate,
            "sweep_launches_timed": sweep_n,
            "roofline_updates_per_ns": peak * 1e3 * 32.0 / per_sw,
            "sweep_share_of_step_time": sweep_ms / total_ms if world == 1 else None}
    if ea3d and "sweep_updates_per_ns" in ea3d:
        p3, h3 = mean_pipes(3, ea3d["timed_betas"])
        ea3d["roofline"] = roofline_record(p3, ea3d["sweep_updates_per_ns"], nsm, f_hz)
        ea3d["roofline"]["zero_class_steps"] = {str(z): c for z, c in sorted(h3.items())}
        ea3d["roofline"]["kernel"] = "k_sweep3d<L,true> (L = 4, 6, 8; grouped replicas)"
    cpu = cpu_mt = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_baseline(64, 5, parallel=False)
        cpu_mt = oracle_baseline(1024, 5, parallel=True)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K,
            "pa_steps_per_s": 1e3 * K / total_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (initial population drawn by the method at beta=0)",
            "config": {"workload": WORKLOAD,
                       "timed_steps": ("all %d steps" % K if K == n_run else
                                       "%d of the %d steps of the five runs, spread evenly "
                                       "(rule, step): %s" % (K, n_run, timed_steps)),
                       "l2": "flushed between timed steps (256 MiB write, outside the step "
                             "events)",
                       "sweep_threads": threads,
                       "parallelism": f"{world} independent runs" if world > 1 else "1 run"},
            "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_mt": cpu_mt, "e2e": e2e,
            "time_to_1e4": acc, "ea3d": ea3d, "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_small(args):
    """Profiling case: one run of --replicas replicas (default 20000) of the benchmark
    lattice, systematic rule; W warm-up steps then K steps, all on one context."""
    import torch
    from paper_2401_07965_gb300 import pa
    betas = np.linspace(0.0, BETA_F, NSTEPS + 1)
    thetas = np.full(NSTEPS, THETA, np.uint32)
    stream = torch.cuda.current_stream()
    p = pa.Population(DIM, L, args.replicas, betas, thetas, "systematic", SEED, stream=stream,
                      sweep_threads=args.threads)
    p.step(args.warmup)
    pa.pa_enable_timing(p.ctx, True)
    p.step(args.steps)
    ms, n, u = pa.pa_sweep_timing(p.ctx)
    print(json.dumps({"case": "small", "R": args.replicas,
                      "threads": pa.pa_get_sweep_threads(p.ctx),
                      "sweep_ms_per_launch": ms / max(n, 1),
                      "sweep_updates_per_ns": u / (ms * 1e6)}), flush=True)
    p.close()
    return 0


def _kaufman(L, beta):
    with open(os.path.join(ROOT, "tests", "golden", "kaufman_lnZ.txt")) as fh:
        for ln in fh:
            if ln.startswith("#"):
                continue
            l, b, v = ln.split()
            if int(l) == L and abs(float(b) - beta) < 1e-12:
                return float(v)
    return None


def _timed_batch(pa, batch, n_steps, stream):
    """Device time of n_steps graph-replayed temperature steps of a batch (CUDA events)."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    batch.step(n_steps)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def _line(workload, value, ms, steps, warmup, extra):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": ms / max(steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def ea3d_batch(pa, stream, realizations=64, steps=20, warmup=5, timed_sweeps=False):
    """The 3D spin-glass batch (L = 4, 6, 8 periodic, `realizations` disorder realizations
    per L from disorder seed 3, R = 50000 each, beta 0 -> 3 in 300 steps, theta = 10,
    systematic): `steps` temperature steps spread evenly over the schedule are timed
    (CUDA events around each graph-replayed step; the runs advance through all 300).
    Returns spin updates/ns of the timed steps (and of the sweep kernels alone)."""
    import torch
    n = 300
    betas = np.linspace(0.0, 3.0, n + 1)
    thetas = np.full(n, 10, np.uint32)
    runs = [{"dim": 3, "L": L, "R": 50000, "couplings": ("ea", 3, 64 * k + r), "ensemble": k}
            for k, L in enumerate((4, 6, 8)) for r in range(realizations)]
    b = pa.Batch(runs, betas, thetas, "systematic", 1000, stream=stream, sweep_threads="auto")
    b.step(warmup)
    first = warmup + 1
    timed = sorted({first + int((k + 0.5) * (n - warmup) / steps) for k in range(steps)})
    timed = [t for t in timed if t <= n]
    upd_step = float(sum(10 * (L ** 3) * 50000 for L in (4, 6, 8)) * realizations)
    ms, sweep_ms, done = 0.0, 0.0, warmup
    for t in timed:
        if t - 1 > done:
            b.step(t - 1 - done)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if timed_sweeps:
            pa.pa_enable_timing(b.ctx, True)
        torch.cuda.synchronize()
        e0.record(stream)
        b.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        if timed_sweeps:
            sm, _, _ = pa.pa_sweep_timing(b.ctx)
            sweep_ms += sm
            pa.pa_enable_timing(b.ctx, False)
        done = t
    R_check = [b.observables(m)["R_i"] for m in (0, realizations, 2 * realizations)]
    b.close()
    out = {"updates_per_ns": upd_step * len(timed) / (ms * 1e6), "ms_per_step": ms / len(timed),
           "timed_steps": timed, "timed_betas": [float(betas[t]) for t in timed],
           "runs": len(runs), "R_i_check": R_check}
    if timed_sweeps:
        out["sweep_updates_per_ns"] = upd_step * len(timed) / (sweep_ms * 1e6)
        out["sweep_share_of_step_time"] = sweep_ms / ms
    return out


def run_ea3d(args):
    """3D Edwards-Anderson +-J, L in {4, 6, 8} periodic, 64 disorder realizations per L
    (couplings iid +-1 from disorder seed 3), R=50000 each, beta 0 -> 3 in 300 steps,
    theta=10, systematic: 192 runs advanced by the same kernels, steps replayed as graphs;
    K steps spread over the schedule are timed."""
    import torch
    from paper_2401_07965_gb300 import pa
    stream = torch.cuda.current_stream()
    K = args.steps if args.steps != 1000 else 30
    res = ea3d_batch(pa, stream, args.realizations, K, args.warmup, timed_sweeps=True)
    _line(f"3D EA +-J, L=4/6/8 x {args.realizations} realizations, R=50000 each, beta 0->3 "
          "in 300 steps, theta=10, systematic", res["updates_per_ns"],
          res["ms_per_step"] * len(res["timed_steps"]), len(res["timed_steps"]), args.warmup,
          {"ea3d": res, "graph": True})
    return 0


def run_weighted(args):
    """2D Ising L=32, beta 0 -> 1 in 150 steps, theta=10, systematic: 256 runs of R=2000 and
    64 of R=8000 in one batch, combined by Eq. (weighted-averages), against one run of
    R=1024000.  Whole runs; free energies compared with Kaufman's exact value."""
    import torch
    from paper_2401_07965_gb300 import pa
    L, n = 32, 150
    betas = np.linspace(0.0, 1.0, n + 1)
    thetas = np.full(n, 10, np.uint32)
    stream = torch.cuda.current_stream()
    runs = [{"dim": 2, "L": L, "R": 2000} for _ in range(256)]
    runs += [{"dim": 2, "L": L, "R": 8000} for _ in range(64)]
    exact = _kaufman(L, 1.0)
    b = pa.Batch(runs, betas, thetas, "systematic", 2000, stream=stream, sweep_threads="auto")
    ms_b = _timed_batch(pa, b, n, stream)
    w = b.weighted(0)[n]
    b.close()
    s = pa.Batch([{"dim": 2, "L": L, "R": 1024000}], betas, thetas, "systematic", 3000,
                 stream=stream, sweep_threads="auto")
    ms_s = _timed_batch(pa, s, n, stream)
    mbf_s, _ = s.free_energy(0)
    s.close()
    upd = 10.0 * L * L * 1024000 * n
    _line("weighted averaging: 256 runs R=2000 + 64 runs R=8000 of 2D Ising L=32 (beta 0->1, "
          "150 steps, theta=10, systematic) in one batch vs one run of R=1024000",
          upd / (ms_b * 1e6), ms_b, n, 0,
          {"batch": {"ms": ms_b, "updates_per_ns": upd / (ms_b * 1e6),
                     "f_err_per_spin": abs(w["minus_beta_F"] - exact) / (L * L),
                     "weighted_c": w["c"], "naive_c": w["c_naive"], "eff_runs": w["eff_runs"]},
           "single": {"ms": ms_s, "updates_per_ns": upd / (ms_s * 1e6),
                      "f_err_per_spin": abs(mbf_s - exact) / (L * L)}})
    return 0


def _spread_thetas(n, sweeps):
    """n per-step sweep numbers, as equal as integers allow, summing to sweeps."""
    base, extra = divmod(int(sweeps), int(n))
    th = np.full(n, base, np.uint32)
    th[np.linspace(0, n - 1, extra).astype(int) if extra else []] += 1
    return th


def _plain_point(pa, L, n, R, thetas, seeds, stream, exact):
    errs, times = [], []
    betas = np.linspace(0.0, 1.0, n + 1)
    for seed in seeds:
        b = pa.Batch([{"dim": 2, "L": L, "R": R}], betas, thetas, "systematic", seed,
                     stream=stream, sweep_threads="auto")
        times.append(_timed_batch(pa, b, n, stream))
        mbf, _ = b.free_energy(0)
        errs.append(abs(mbf - exact) / (L * L))
        b.close()
    return {"R": R, "steps": n, "sweeps": int(np.sum(thetas)), "ms": float(np.mean(times)),
            "max_err_per_spin": float(max(errs))}


def _batch_point(pa, L, n, M, Rm, theta, seeds, stream, exact):
    """M runs of Rm replicas in one batch (one launch per phase, graph replay), combined by
    Eq. (weighted-averages): ln Z = ln(sum_m R_m Z_m / sum_m R_m)."""
    errs, times = [], []
    betas = np.linspace(0.0, 1.0, n + 1)
    for seed in seeds:
        b = pa.Batch([{"dim": 2, "L": L, "R": Rm, "ensemble": 0} for _ in range(M)], betas,
                     np.full(n, theta, np.uint32), "systematic", seed, stream=stream,
                     sweep_threads="auto")
        times.append(_timed_batch(pa, b, n, stream))
        w = b.weighted(0)[n]
        errs.append(abs(w["minus_beta_F"] - exact) / (L * L))
        b.close()
    return {"R": Rm * M, "runs": M, "R_per_run": Rm, "steps": n, "sweeps": n * theta,
            "ms": float(np.mean(times)), "max_err_per_spin": float(max(errs))}


def _learned_point(pa, CT, L, K, R, budget, seeds, stream, exact, bits):
    errs, times = [], []
    for seed in seeds:
        pop = CT.controlled_run(2, L, ("ferro",), R, np.linspace(0.0, 1.0, K + 1), 4, 10, bits,
                                seed=seed, budget=budget, stream=stream, sweep_threads="auto")
        times.append(_chunked(pa, pop, stream, K))
        mbf, _ = pop.free_energy()
        errs.append(abs(mbf - exact) / (L * L))
        pop.close()
    return {"R": R, "grid": K, "sweeps": budget, "ms": float(np.mean(times)),
            "max_err_per_spin": float(max(errs))}


def _best(grid, target=1e-4):
    ok = [g for g in grid if g["max_err_per_spin"] <= target]
    return min(ok, key=lambda g: g["ms"]) if ok else None


def accuracy_l64(pa, dev, seeds=(11, 12, 13, 14, 15)):
    """Time to a free energy within 1e-4 per spin of Kaufman's exact value at beta_f = 1 on
    the benchmark lattice (2D Ising L=64), systematic rule, worst of 5 seeds, device time
    per run (CUDA events, graph replay): the least time over
      plain:      200 equal steps, R in {3000, R1, 10^4, 3 10^4, 10^5} x theta in {2, 5, 10};
      plain800:   800 equal steps (the learned schedule's grid) at 1000 or 2000 sweeps in
                  all, R in {3000, R1, 10^4, 3 10^4};
      batched:    M in {4, 8, 12} runs of 2500 replicas, 4 of 7500, or 4 and 8 of R1/4 in
                  one batch, 200 steps, theta in {2, 5, 10}, combined by Eq.
                  (weighted-averages);
      learned:    the learned controller on the 800-point grid, budgets 500, 1000, 1500 or
                  2000 sweeps, R in {3000, R1, 10^4, 3 10^4}.
    R1 = 32 x the GPU's SM count (4864 on a GB300): one replica group per SM, the largest
    population whose sweep is one wave of CTAs."""
    import torch
    from paper_2401_07965_gb300 import controller as CT
    stream = torch.cuda.Stream(dev)
    Lx = 64
    exact = _kaufman(Lx, 1.0)
    out = {"target_per_spin": 1e-4, "seeds": len(seeds), "lattice": "2D Ising L=64, beta 0->1",
           "what": "device ms per run of the cheapest configuration whose worst-seed |f - f_exact| "
                   "per spin is <= 1e-4 (Kaufman's exact finite-lattice value)"}
    R1 = 32 * torch.cuda.get_device_properties(dev).multi_processor_count
    out["R1"] = R1
    plain = [_plain_point(pa, Lx, 200, R, np.full(200, th, np.uint32), seeds, stream, exact)
             for R in (3000, R1, 10000, 30000, 100000) for th in (2, 5, 10)]
    p800 = [_plain_point(pa, Lx, 800, R, _spread_thetas(800, sw), seeds, stream, exact)
            for R in (3000, R1, 10000, 30000) for sw in (1000, 2000)]
    batched = [_batch_point(pa, Lx, 200, M, Rm, th, seeds, stream, exact)
               for M, Rm in ((4, 2500), (8, 2500), (12, 2500), (4, 7500), (4, R1 // 4),
                             (8, R1 // 4)) for th in (2, 5, 10)]
    out["plain"] = {"best": _best(plain), "grid": plain}
    out["plain800"] = {"best": _best(p800), "grid": p800}
    out["batched"] = {"best": _best(batched), "grid": batched,
                      "what": "M runs of R/M replicas in one batch, combined by Eq. "
                              "(weighted-averages), 200 steps"}
    if os.path.exists(CT.WEIGHTS):
        bits = CT.load()
        learned = [_learned_point(pa, CT, Lx, 800, R, bud, seeds, stream, exact, bits)
                   for R in (3000, R1, 10000, 30000) for bud in (500, 1000, 1500, 2000)]
        out["learned"] = {"best": _best(learned), "grid": learned}
    cands = [v["best"] for k, v in out.items() if isinstance(v, dict) and v.get("best")]
    bp = [out[k]["best"] for k in ("plain", "plain800") if out[k]["best"]]
    out["best_plain_ms"] = min(g["ms"] for g in bp) if bp else None
    out["best_batched_ms"] = out["batched"]["best"]["ms"] if out["batched"]["best"] else None
    out["best_learned_ms"] = (out["learned"]["best"]["ms"]
                              if out.get("learned", {}).get("best") else None)
    out["value_ms"] = min(g["ms"] for g in cands) if cands else None
    return out


def run_accuracy(args):
    """Time to a free energy within 1e-4 per spin of Kaufman's value at beta_f = 1: the L=64
    grids of the headline line's time_to_1e4 record, plus the 2D Ising L=16 lattice (100
    steps, grid over R and theta).  Value: the L=64 figure."""
    import torch
    from paper_2401_07965_gb300 import pa
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(dev)
    exact16 = _kaufman(16, 1.0)
    g16 = [_plain_point(pa, 16, 100, R, np.full(100, th, np.uint32), (11, 12, 13, 14, 15),
                        stream, exact16)
           for R in (1000, 3000, 10000, 30000) for th in (2, 5, 10)]
    acc = accuracy_l64(pa, dev)
    acc["L16"] = {"best": _best(g16), "grid": g16}
    # the weighted-averaging lattice, L=32 with 150 steps: single runs against batches
    exact32 = _kaufman(32, 1.0)
    seeds = (11, 12, 13, 14, 15)
    g32 = [_plain_point(pa, 32, 150, R, np.full(150, th, np.uint32), seeds, stream, exact32)
           for R in (2000, 8000, 32000) for th in (2, 5, 10)]
    b32 = [_batch_point(pa, 32, 150, M, Rm, th, seeds, stream, exact32)
           for M, Rm in ((8, 2000), (16, 2000), (4, 8000)) for th in (2, 5)]
    acc["L32"] = {"plain": {"best": _best(g32), "grid": g32},
                  "batched": {"best": _best(b32), "grid": b32}}
    v = acc["value_ms"]
    _line("time to |f - f_exact| <= 1e-4 per spin at beta=1, 2D Ising L=64 (plain 200 or 800 "
          "steps, learned schedule) and L=16 (100 steps), systematic, worst of 5 seeds",
          v, v or 0.0, 200, 0, {"unit": "ms", "higher_is_better": False, "results": acc})
    return 0


def _chunked(pa, pop, stream, n_max, chunk=16):
    """Advance a run in chunks of steps until n_max steps or, under the controller, until
    beta_f; device time summed over the chunks (CUDA events on the run's stream)."""
    import torch
    ms = 0.0
    done = 0
    while done < n_max:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = min(chunk, n_max - done)
        a.record(stream)
        try:
            pop.step(k)
        except pa.PAError as e:
            if e.status != pa.PA_ERR_DONE:
                raise
            b.record(stream)
            torch.cuda.synchronize()
            break
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        done += k
        pa.pa_sync(pop.ctx)
    return ms


def _schedule_arm(pa, CT, sysdef, seeds, stream, plain=None, learned=None, bits=None):
    """Runs of one schedule over seeds: plain = (n_steps, theta); learned = (grid points K,
    plain_units, plain_theta, budget).  Returns per-seed -beta F, e, rho_t / R, ms, steps."""
    dim, L, cpl, R, bf = sysdef
    out = []
    for seed in seeds:
        if plain:
            n, theta = plain
            pop = pa.Population(dim, L, R, np.linspace(0.0, bf, n + 1),
                                np.full(n, theta, np.uint32), "systematic", seed,
                                couplings=cpl, stream=stream, sweep_threads="auto")
            ms = _chunked(pa, pop, stream, n)
            sweeps = n * theta
        else:
            K, units, theta, budget = learned
            pop = CT.controlled_run(dim, L, cpl, R, np.linspace(0.0, bf, K + 1), units, theta,
                                    bits, seed=seed, budget=budget, stream=stream,
                                    sweep_threads="auto")
            ms = _chunked(pa, pop, stream, K)
            _, th = pa.pa_schedule_taken(pop.ctx, K + 1)
            sweeps = int(th.sum())
        o = pop.observables()
        out.append({"mbf": L ** dim * math.log(2.0) + o["sum_lnQ"], "e": o["e"],
                    "rho": o["rho_t"] / R, "ms": ms, "steps": o["step"], "sweeps": sweeps})
        pop.close()
    return out


def _boot_rms(err, rng, nboot=2000):
    """Bootstrap (over seeds) standard error of the root-mean-square of err."""
    idx = rng.integers(0, len(err), size=(nboot, len(err)))
    return float(np.sqrt((err[idx] ** 2).mean(axis=1)).std(ddof=1))


def _summ(rows, ref_mbf, ref_e, N, rng):
    err = np.array([(r["mbf"] - ref_mbf) / N for r in rows])
    ms = np.array([r["ms"] for r in rows])
    out = {"rms_f_err_per_spin": float(np.sqrt(np.mean(err ** 2))),
           "rms_se": _boot_rms(err, rng),
           "mean_f_err_per_spin": float(err.mean()),
           "mean_se": float(err.std(ddof=1) / np.sqrt(len(err))),
           "rho_t_over_R": float(np.mean([r["rho"] for r in rows])),
           "ms": float(ms.mean()), "ms_se": float(ms.std(ddof=1) / np.sqrt(len(ms))),
           "steps": float(np.mean([r["steps"] for r in rows])),
           "sweeps": float(np.mean([r["sweeps"] for r in rows])), "seeds": len(rows)}
    if ref_e is not None:
        out["rms_e_err"] = float(np.sqrt(np.mean([(r["e"] - ref_e) ** 2 for r in rows])))
    out["_err"] = err
    return out


def _compare(arm, plain, rng, nboot=2000):
    """Learned arm against the plain arm (independent seeds): the difference of the rms
    errors with its bootstrap standard error, and whether the learned arm is better (or
    not worse) by more than two standard errors."""
    a, b = arm["_err"], plain["_err"]
    ia = rng.integers(0, len(a), size=(nboot, len(a)))
    ib = rng.integers(0, len(b), size=(nboot, len(b)))
    d = np.sqrt((a[ia] ** 2).mean(axis=1)) - np.sqrt((b[ib] ** 2).mean(axis=1))
    diff = arm["rms_f_err_per_spin"] - plain["rms_f_err_per_spin"]
    se = float(d.std(ddof=1))
    return {"rms_diff": diff, "rms_diff_se": se,
            "better_by_2se": bool(diff < -2 * se), "worse_by_2se": bool(diff > 2 * se),
            "time_ratio": arm["ms"] / plain["ms"]}


def run_controller(args):
    """The learned schedule controller against the plain schedule, with bootstrap errors.

    3D +-J spin glass L=10 (disorder seed 5, realization 0), R=100000, beta 0 -> 3: plain 300
    steps of 10 sweeps against the learned schedule on a 600-point grid with the same 3000
    sweeps, and with 2250 and 1500; errors against the mean of four R=10^6 runs (600 steps,
    30 sweeps; no exact value exists).  2D Ising L=64, R=10000, beta 0 -> 1: plain 200 steps
    of 10 sweeps against the learned schedule on an 800-point grid with 2000, 1500 and 1000
    sweeps; errors against Kaufman's exact free energy.  --seeds independent seeds per arm.
    Value: device time of the cheapest learned schedule whose rms free-energy error (3D EA
    L=10) is not worse than the plain schedule's by two bootstrap standard errors."""
    import torch
    from paper_2401_07965_gb300 import controller as CT
    from paper_2401_07965_gb300 import pa
    if not os.path.exists(CT.WEIGHTS):
        print(json.dumps({"metric": METRIC, "value": None, "unavailable":
                          "no trained controller weights"}), flush=True)
        return 1
    bits = CT.load()
    stream = torch.cuda.Stream()
    if args.case == "small":
        # profiling case: two learned runs of the time-to-1e-4 arm (2D Ising L=64,
        # R=3000, 800-point grid, 2000 sweeps, 512 sweep threads), device time per run
        ms = []
        for seed in (11, 12):
            pop = CT.controlled_run(2, 64, ("ferro",), 3000, np.linspace(0.0, 1.0, 801), 4, 10,
                                    bits, seed=seed, budget=2000, stream=stream,
                                    sweep_threads=512)
            ms.append(_chunked(pa, pop, stream, 800))
            pop.close()
        _line("learned schedule, profiling case: 2D Ising L=64, R=3000, 800-point grid, "
              "2000 sweeps, 2 seeds", float(np.mean(ms)), float(np.sum(ms)), 2, 0,
              {"unit": "ms per run", "higher_is_better": False})
        return 0
    rng = np.random.default_rng(2024)
    S = args.seeds
    seeds = range(1, S + 1)
    res = {}
    # spin glass, config of the learned-schedule benchmark
    ea = (3, 10, ("ea", 5, 0), 100000, 3.0)
    refs = _schedule_arm(pa, CT, (3, 10, ("ea", 5, 0), 1000000, 3.0), [4242, 4243, 4244, 4245],
                         stream, plain=(600, 30))
    ref_mbf = float(np.mean([r["mbf"] for r in refs]))
    ref_e = float(np.mean([r["e"] for r in refs]))
    N = 1000
    res["ea10"] = {"reference": {"R": 1000000, "runs": len(refs), "steps": 600, "theta": 30,
                                 "mbf": ref_mbf, "mbf_se": float(np.std([r["mbf"] for r in refs],
                                                                        ddof=1) / 2.0),
                                 "e": ref_e, "ms": float(np.mean([r["ms"] for r in refs]))}}
    res["ea10"]["plain"] = _summ(_schedule_arm(pa, CT, ea, seeds, stream, plain=(300, 10)),
                                 ref_mbf, ref_e, N, rng)
    for budget in (3000, 2250, 1500):
        res["ea10"][f"learned_{budget}"] = _summ(
            _schedule_arm(pa, CT, ea, seeds, stream, learned=(600, 2, 10, budget), bits=bits),
            ref_mbf, ref_e, N, rng)
    # 2D Ising, exact reference
    L = 64
    exact = _kaufman(L, 1.0)
    ising = (2, L, ("ferro",), 10000, 1.0)
    res["ising64"] = {"plain": _summ(_schedule_arm(pa, CT, ising, seeds, stream,
                                                   plain=(200, 10)), exact, None, L * L, rng)}
    for budget in (2000, 1500, 1000):
        res["ising64"][f"learned_{budget}"] = _summ(
            _schedule_arm(pa, CT, ising, seeds, stream, learned=(800, 4, 10, budget), bits=bits),
            exact, None, L * L, rng)
    for sysname in ("ea10", "ising64"):
        plain = res[sysname]["plain"]
        for key in list(res[sysname]):
            if key.startswith("learned_"):
                res[sysname][key]["vs_plain"] = _compare(res[sysname][key], plain, rng)
    for sysname in ("ea10", "ising64"):
        for key, arm in res[sysname].items():
            arm.pop("_err", None)
    p_ea = res["ea10"]["plain"]
    ok = [res["ea10"][f"learned_{b}"] for b in (3000, 2250, 1500)
          if not res["ea10"][f"learned_{b}"]["vs_plain"]["worse_by_2se"]]
    best = min(ok, key=lambda r: r["ms"]) if ok else None
    _line("learned vs plain schedule: 3D EA +-J L=10, R=100000, beta 0->3, plain 300 steps x "
          "10 sweeps vs learned on a 600-point grid at 3000/2250/1500 sweeps; 2D Ising L=64, "
          f"R=10000, beta 0->1 vs Kaufman; {S} seeds each, bootstrap standard errors",
          best["ms"] if best else None, best["ms"] if best else 0.0, 0, 0,
          {"unit": "ms", "higher_is_better": False,
           "what": "device ms per run of the cheapest learned schedule whose rms free-energy "
                   "error (3D EA L=10) is not worse than the plain 3000-sweep schedule's by two "
                   "bootstrap standard errors",
           "plain_ms": p_ea["ms"], "results": res})
    return 0


def run_overlap(args):
    """Overlap distribution P(q) of the 2D +-J spin glass, L=32 (the lattice of the paper's
    P(q) figures): 16 disorder samples (disorder seed 3) x 2 independent populations of
    R=100000, beta 0 -> 3 in 100 steps, theta=25, systematic, in one batch; then the
    overlap kernel over the 16 run pairs, timed alone with CUDA events (L2 flushed between
    calls, outside the events) against the measured HBM bandwidth."""
    import torch
    from paper_2401_07965_gb300 import pa
    L, R, n, S = 32, 100000, 100, 16
    if args.case == "small":
        n = 10  # profiling: a short anneal before the same overlap launch
    N = L * L
    betas = np.linspace(0.0, 3.0, n + 1)
    thetas = np.full(n, 25, np.uint32)
    runs = [{"dim": 2, "L": L, "R": R, "couplings": ("ea", 3, s), "ensemble": s}
            for s in range(S) for _ in range(2)]
    stream = torch.cuda.Stream()
    b = pa.Batch(runs, betas, thetas, "systematic", 3000, stream=stream, sweep_threads="auto")
    ms_anneal = _timed_batch(pa, b, n, stream)
    pairs = [(2 * s, 2 * s + 1) for s in range(S)]
    hist = torch.empty((S, N + 1), dtype=torch.int32, device="cuda")
    P = pa.pa_overlap(b.ctx, [p[0] for p in pairs], [p[1] for p in pairs], hist.data_ptr(), N)
    # the rows of the 32 populations (410 MB) exceed the 129 MB L2, so back-to-back calls
    # read them from HBM; timing a burst of calls keeps the host's enqueue time out of the
    # device time
    times = []
    reps = max(args.steps if args.steps != 1000 else 20, 3)
    run_a, run_b = [p[0] for p in pairs], [p[1] for p in pairs]
    for k in range(args.warmup):
        pa.pa_overlap(b.ctx, run_a, run_b, hist.data_ptr(), N, weighted=False)
    for k in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            pa.pa_overlap(b.ctx, run_a, run_b, hist.data_ptr(), N, weighted=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / reps)
    h = hist.cpu().numpy().view(np.uint32)
    b.close()
    ms = statistics.median(times)
    Wp = ((N + 31) // 32 + 3) // 4 * 4
    bytes_alg = 2.0 * S * R * Wp * 4
    peaks, src = _peaks()
    gbs = bytes_alg / (ms * 1e6)
    q = 1.0 - 2.0 * np.arange(N + 1) / N
    q2 = float((P * q * q).sum())
    _line("overlap distribution P(q): 2D +-J L=32, 16 samples x 2 populations of R=100000, "
          "beta 0->3 in 100 steps, theta=25, systematic; overlap kernel over the 16 pairs",
          gbs, ms * reps, reps, args.warmup,
          {"unit": "GB/s", "what": "algorithmic bytes (2 rows of 128 B per replica pair) / "
                                   "device time per call of the overlap entry point (median "
                                   "of 5 bursts of back-to-back calls)",
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
                        "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                        "kernel": "k_overlap_hist", "peak_source": f"hbm_gbs ({src})"},
           "anneal_ms": ms_anneal,
           "anneal_updates_per_ns": 25.0 * N * R * 2 * S * n / (ms_anneal * 1e6),
           "weighted_q2": q2, "P_q0": float(P[N // 2]),
           "pairs_per_sample": [int(x) for x in h.sum(axis=1)[:3]],
           "l2": "not flushed: the 410 MB of rows read per call exceed the 129 MB L2"})
    return 0


def run_partial(args):
    """Partial resampling (resample only when the effective size of the reweighted
    population falls below alpha R) against resampling at every step: 2D Ising L=64,
    R=10000, beta 0 -> 1 in 200 steps, theta=10, systematic, 5 seeds per arm; device time
    per run (graph replay), resampling steps, free-energy error against Kaufman's value."""
    import torch
    from paper_2401_07965_gb300 import pa
    L, R, n = 64, 10000, 200
    betas = np.linspace(0.0, 1.0, n + 1)
    thetas = np.full(n, 10, np.uint32)
    exact = _kaufman(L, 1.0)
    stream = torch.cuda.Stream()
    arms = {}
    for alpha in (None, 0.9, 0.5, 0.2):
        ms, errs, res = [], [], []
        for seed in (21, 22, 23, 24, 25):
            b = pa.Batch([{"dim": 2, "L": L, "R": R}], betas, thetas, "systematic", seed,
                         stream=stream, sweep_threads="auto")
            if alpha is not None:
                b.set_partial_resampling(alpha)
            ms.append(_timed_batch(pa, b, n, stream))
            mbf, _ = b.free_energy(0)
            errs.append((mbf - exact) / (L * L))
            res.append(sum(r["resampled"] for r in b.trace(0)[1:]))
            b.close()
        arms["every step" if alpha is None else f"alpha={alpha}"] = {
            "ms": float(np.mean(ms)), "rms_f_err_per_spin": float(np.sqrt(np.mean(np.square(errs)))),
            "max_f_err_per_spin": float(np.max(np.abs(errs))),
            "resampling_steps": float(np.mean(res))}
    base = arms["every step"]
    _line("partial resampling: 2D Ising L=64, R=10000, beta 0->1 in 200 steps, theta=10, "
          "systematic, 5 seeds; alpha = 0.9 / 0.5 / 0.2 against every step",
          10.0 * L * L * R * n / (arms["alpha=0.5"]["ms"] * 1e6), arms["alpha=0.5"]["ms"], n, 0,
          {"what": "spin updates/ns of a whole run with alpha = 0.5 (graph replay)",
           "every_step_updates_per_ns": 10.0 * L * L * R * n / (base["ms"] * 1e6),
           "arms": arms})
    return 0


def run_split(args):
    """Where a temperature step's time goes: 2D Ising L=64, beta 0 -> 1 in 200 steps, for
    R = 3000 / 30000 / 100000 (theta = 10 / 5 / 10) and three copy-count rules; the whole
    run replayed as graphs (device time of all 200 steps, CUDA events) against the sweep
    kernel alone (its launches timed by the library's own events in a second run of the
    same seed).  outside_sweep = 1 - sweep time / step time."""
    import torch
    from paper_2401_07965_gb300 import pa
    n = 200
    betas = np.linspace(0.0, 1.0, n + 1)
    stream = torch.cuda.Stream()
    out = {}
    for rule in ("systematic", "nearest", "multinomial"):
        for R, th in ((3000, 10), (30000, 5), (100000, 10)):
            thetas = np.full(n, th, np.uint32)
            b = pa.Batch([{"dim": 2, "L": 64, "R": R}], betas, thetas, rule, 11, stream=stream)
            ms = _timed_batch(pa, b, n, stream)
            b.close()
            p = pa.Population(2, 64, R, betas, thetas, rule, 11, stream=stream)
            pa.pa_enable_timing(p.ctx, True)
            p.step(n)
            sms, cnt, _ = pa.pa_sweep_timing(p.ctx)
            p.close()
            out[f"{rule} R={R} theta={th}"] = {
                "us_per_step": 1e3 * ms / n, "sweep_us_per_step": 1e3 * sms / cnt,
                "outside_sweep": 1.0 - (sms / cnt) / (ms / n)}
    key = "systematic R=30000 theta=5"
    _line("step split: 2D Ising L=64, beta 0->1 in 200 steps; R = 3000 / 30000 / 100000, "
          "systematic / nearest / multinomial", out[key]["outside_sweep"],
          out[key]["us_per_step"] * n / 1e3, n, 0,
          {"unit": "fraction of step time outside the sweep kernel",
           "higher_is_better": False, "what": key, "split": out})
    return 0


def run_e2e(args, pa, stream, seed, dev, threads=0):
    """Whole runs through the C ABI: host schedule -> pa_init -> per step pa_step +
    pa_observables (device -> host) -> pa_free_energy.  Host wall clock."""
    import ctypes as C
    import torch
    betas = np.linspace(0.0, BETA_F, NSTEPS + 1)
    thetas = np.full(NSTEPS, THETA, np.uint32)
    n_total = max(args.steps, NSTEPS * len(RULES))   # whole runs of the five rules
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    updates = 0.0
    done = 0
    r = 0
    h2d = 0
    d2h = 0
    while done < n_total:
        rule = RULES[r % 5]
        n = min(NSTEPS, n_total - done)
        ctx = pa.pa_init(DIM, L, ("ferro",), R, 0, betas, thetas, pa.RESAMPLERS[rule], seed,
                         stream.cuda_stream)
        if threads:
            pa.pa_set_sweep_threads(ctx, threads)
        h2d += betas.nbytes + thetas.nbytes + 3 * 8 * NSTEPS + 16 * NSTEPS
        for _ in range(n):
            pa.pa_step(ctx, 1)
            o = pa.pa_observables(ctx)
            d2h += C.sizeof(pa.pa_obs)
            updates += THETA * L * L * o["R_i"]
        pa.pa_free_energy(ctx)
        pa.pa_destroy(ctx)
        done += n
        r += 1
    sec = time.perf_counter() - t0
    return {"value": updates / (sec * 1e9), "unit": UNIT,
            "h2d_bytes_per_step": h2d / n_total, "d2h_bytes_per_step": d2h / n_total,
            "what": "pa_init from host arrays, then pa_step + pa_observables per step, "
                    "pa_free_energy per run; host wall clock including init"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the time-to-1e-4 sub-record of the headline line")
    ap.add_argument("--no-ea3d", action="store_true",
                    help="skip the batched 3D spin-glass sub-record of the headline line")
    ap.add_argument("--threads", type=int, default=0, help="small case: sweep threads per CTA")
    ap.add_argument("--replicas", type=int, default=20000, help="small case: population size")
    ap.add_argument("--realizations", type=int, default=64,
                    help="ea3d workload: disorder realizations per lattice size")
    ap.add_argument("--seeds", type=int, default=24, help="controller workload: seeds per arm")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: one run of R=20000 replicas of the same lattice (profiling)")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "ea3d", "weighted", "accuracy", "controller",
                             "overlap", "partial", "split"],
                    help="headline: the benchmark line; ea3d / weighted: the batched "
                         "workloads; accuracy: time to a free energy within 1e-4 per spin; "
                         "controller: learned against plain schedule; overlap: P(q) of "
                         "two populations per spin-glass sample; partial: resampling only "
                         "when the weights' effective size is low; split: step time "
                         "outside the sweep kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "small" and args.workload == "headline":
        return run_small(args)
    if args.workload == "ea3d":
        return run_ea3d(args)
    if args.workload == "weighted":
        return run_weighted(args)
    if args.workload == "accuracy":
        return run_accuracy(args)
    if args.workload == "controller":
        return run_controller(args)
    if args.workload == "overlap":
        return run_overlap(args)
    if args.workload == "partial":
        return run_partial(args)
    if args.workload == "split":
        return run_split(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
