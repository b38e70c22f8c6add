"""Multi-rank host logic on CPU (gloo, world size 2): surfaces are sharded
without data exchange, the shards cover every surface exactly once, and the
bench's timing is the maximum over ranks."""
import os
import socket

import pytest

from paper_2603_28160_gb300 import shard
from paper_2603_28160_gb300 import workloads as W


def test_split_by_cost_is_a_balanced_partition():
    costs = [w.process.cells for w in W.lhs_batch(n=257, seed=3)]
    for world in (1, 2, 3, 8):
        parts = shard.split_by_cost(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
        assert parts == shard.split_by_cost(costs, world)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = [w.process.cells for w in W.lhs_batch(n=64, seed=9)]
    mine = shard.split_by_cost(costs, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)  # per-rank step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    q.put((rank, gathered, float(t.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_overlap():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, tmax in results:
        assert tmax == 2.0
        a, b = gathered
        assert not set(a) & set(b)
        assert sorted(a + b) == list(range(64))
