"""Host logic of the multi-GPU path on CPU: longest-processing-time-first
partition of independent instances and the max / sum gathers over ranks
(gloo, world size 2). No GPU and no data-path collective are involved."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2103_05857_gb300.shard import gather_max, gather_sum, lpt_partition


def test_lpt_partition_covers_and_balances():
    work = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4]
    parts = lpt_partition(work, 3)
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(work)))
    loads = [sum(work[k] for k in p) for p in parts]
    # LPT is within 4/3 of the optimum; here the total 48 splits 16/16/16
    assert max(loads) <= 4 / 3 * (sum(work) / 3) + max(work)
    assert loads == [16, 16, 16]
    assert lpt_partition(work, 1) == [list(range(len(work)))]
    assert lpt_partition([], 2) == [[], []]
    with pytest.raises(ValueError):
        lpt_partition(work, 0)


def test_lpt_partition_deterministic_ties():
    assert lpt_partition([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        work = [(17 * k) % 23 + 1 for k in range(40)]
        parts = lpt_partition(work, world)
        mine = parts[rank]
        # each rank "solves" its share: the timing is its share's load
        t = float(sum(work[k] for k in mine))
        q.put((rank, mine, gather_max(t, world), gather_sum(len(mine), world)))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_partition_and_gather():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    work = [(17 * k) % 23 + 1 for k in range(40)]
    shares = [o[1] for o in out]
    assert sorted(shares[0] + shares[1]) == list(range(40))
    assert not set(shares[0]) & set(shares[1])
    loads = [sum(work[k] for k in s) for s in shares]
    assert all(o[2] == max(loads) for o in out)   # max over ranks
    assert all(o[3] == 40 for o in out)           # sum over ranks
