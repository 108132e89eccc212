"""Runs on several GPUs, one process per GPU (torch.distributed).

Population annealing needs no data exchange between independent runs: each
rank advances its own runs with its own seeds, and only at the end are the
runs combined with the weighted averages of Sec. 4 (Eq. weighted-averages).
gather_rows collects every run's summary at one step (population size, sum of
ln Q, exact sums: a pa_run_row of 80 bytes) from all ranks; combine then forms
the weighted averages on rank 0's GPU with pa_weighted_rows.  Any backend that
supports all_gather_object works (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

from . import pa


def gather_rows(local_rows, group=None):
    """All ranks' rows, in rank order and then in each rank's own order, on every rank."""
    import torch.distributed as dist
    payload = [bytes(r) for r in local_rows]
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, payload, group=group)
    return [pa.pa_run_row.from_buffer_copy(b) for part in parts for b in part]


def combine(local_rows, N, beta, step=0, group=None, stream=0):
    """Weighted averages over the runs of all ranks at one step; the result on rank 0
    (None elsewhere)."""
    import torch.distributed as dist
    rows = gather_rows(local_rows, group)
    if dist.get_rank(group) != 0:
        return None
    return pa.pa_weighted_rows(rows, N, beta, step, stream)
