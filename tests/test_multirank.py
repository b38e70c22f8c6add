"""Multi-rank host logic on CPU (gloo, world size 2): surfaces are sharded
without data exchange, the shards cover every surface exactly once, and the
bench's timing is the maximum over ranks; one surface split in row bands over
ranks gives the whole map's rows and, through two all-reduces of moment
partials, the whole map's roughness."""
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


# --------------------------------------------------------------------------
# One surface in row bands over two ranks: each rank predicts its band (here
# with the oracle, on the CPU), the bands equal the whole map's rows, and the
# roughness merged from the bands' moment partials by two all-reduces equals
# the whole map's.
# --------------------------------------------------------------------------
def _np_partials(H, about):
    import numpy as np
    if H.size == 0:
        return list(shard.EMPTY_PARTIALS)
    d = H - about
    return [float(H.size), float(d.sum()), float(H.min()), float(H.max()), float(np.abs(d).sum()),
            float((d * d).sum()), float((d ** 3).sum()), float((d ** 4).sum())]


def _band_workload():
    return W.raster_ball_d10(precision="fp64", width=0.3, pitch=0.002, n_passes=3, n_edge=40, rot_step_deg=1.0)


def _band_worker(rank, world, port, q):
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _band_workload()
    k0, k1 = shard.row_bands(w.process.ny, world)[rank]
    band = W.Workload(w.name, w.tool, shard.band_process(w.process, k0, k1))
    Hb = O.fsm(band).H
    rough = shard.distributed_roughness(lambda about: _np_partials(Hb, about), about0=0.0)
    dist.barrier()
    q.put((rank, k0, k1, Hb, rough))
    dist.destroy_process_group()


def test_row_bands_cover_the_map():
    for ny in (1, 5, 200, 201):
        for world in (1, 2, 3, 8):
            bands = shard.row_bands(ny, world)
            assert bands[0][0] == 0 and bands[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(bands, bands[1:]))
            sizes = [k1 - k0 for k0, k1 in bands]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_merge_row_band_roughness(oracle_mod):
    import multiprocessing as mp

    import numpy as np
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted([q.get(timeout=300) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    full = oracle_mod.fsm(_band_workload())
    ok = ~full.flags
    for rank, k0, k1, Hb, rough in results:
        # the band is the whole map's rows
        assert np.array_equal(Hb[ok[k0:k1]], full.H[k0:k1][ok[k0:k1]])
        ref = oracle_mod.roughness(full.H)
        for k in ("n", "mean", "zmin", "zmax", "Sz"):
            assert abs(rough[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), (k, rough[k], ref[k])
        for k in ("Sa", "Sq", "Ssk", "Sku"):
            assert abs(rough[k] - ref[k]) <= 1e-11 * abs(ref[k]), (k, rough[k], ref[k])
    assert results[0][4] == results[1][4]  # every rank gets the same record
