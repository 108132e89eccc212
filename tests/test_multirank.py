"""The N > 1 host path of bench.py on CPU ranks (gloo, world size 2).

Runs on several GPUs are independent populations (replicas only): the ranks
exchange nothing on the data path, and the whole-job figures are the maximum
of the ranks' device times and the sum of their units.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    units = [1.0e9, 3.0e9][rank]
    out[rank] = (bench.combine_over_ranks(ms, units, "cpu"), bench.rank_seed(rank))
    dist.destroy_process_group()


def test_combine_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        (ms, units), seed = res[r]
        assert ms == 20.0 and units == 4.0e9
    assert res[0][1] != res[1][1]


def _rows_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2401_07965_gb300 import distributed as D
    from paper_2401_07965_gb300 import pa
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank advances its own small runs (the oracle stands in for the GPU here)
    L, n = 4, 6
    betas = np.linspace(0.0, 1.0, n + 1)
    rows = []
    for k in range(rank + 1):
        run = O.Run(2, L, O.ferro_couplings(2, L), 50 + 10 * k, betas, np.full(n, 2, np.uint32),
                    O.RESAMPLERS["systematic"], 100 * rank + k)
        for _ in range(n):
            run.step()
        rows.append(pa.run_row(run.obs(), 50 + 10 * k))
    got = D.gather_rows(rows)
    out[rank] = [(r.R_i, r.R, r.sum_lnQ, r.sumE, r.sumE2) for r in got]
    dist.destroy_process_group()


def test_gather_run_rows_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rows_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    # every rank sees rank 0's one run, then rank 1's two runs
    assert res[0] == res[1] and len(res[0]) == 3
    assert [r[1] for r in res[0]] == [50, 50, 60]


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0
