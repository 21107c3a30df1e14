"""Host-side partition of independent instances across ranks (one process
per GPU). A single solve does not shard: every block update reads the
residual the previous one wrote. Independent instances do: each rank solves
its share with no data-path collective; only timings and results are
gathered on the host.
"""
from __future__ import annotations


def lpt_partition(work, nparts):
    """Longest-processing-time-first assignment: instances sorted by work
    (descending, ties by index) go one at a time to the least loaded part
    (ties to the lowest part). Returns a list of index lists, each in
    ascending instance order."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    order = sorted(range(len(work)), key=lambda k: (-work[k], k))
    load = [0] * nparts
    parts = [[] for _ in range(nparts)]
    for k in order:
        p = min(range(nparts), key=lambda q: (load[q], q))
        parts[p].append(k)
        load[p] += work[k]
    return [sorted(p) for p in parts]


def gather_max(value, world_size):
    """Max over ranks of a host float (identity without a process group)."""
    if world_size == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_sum(value, world_size):
    """Sum over ranks of a host float (identity without a process group)."""
    if world_size == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
