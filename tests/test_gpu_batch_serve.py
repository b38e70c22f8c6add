"""Batched and served prediction: one persistent launch over many surfaces of
mixed tools, grids and precisions (also replayed as a CUDA graph), and the
request server with continuous batching -- every result must equal the same
surface predicted alone."""
import time

import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import compare_maps

pytestmark = pytest.mark.gpu


def small_mix(n=14, seed=21):
    ws = W.lhs_batch(n=n, seed=seed, n_edge=40, rot_step_deg=0.5, side_range=(0.15, 0.45),
                     pitch_range_um=(2.0, 6.0))
    return W.mixed_precision(ws, fp64_fraction=0.4, seed=seed)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    ws = small_mix()
    alone = []
    for w in ws:
        out = F.predict(w, ctx)
        torch.cuda.synchronize()
        alone.append((out, ctx.roughness(out)))
    return F, ctx, ws, alone


def rough_array(F, buf, n):
    raw = buf.cpu().numpy().tobytes()
    sz = F.ROUGH_BYTES
    return [F.rough_dict(F.RoughnessOut.from_buffer_copy(raw[i * sz:(i + 1) * sz])) for i in range(n)]


def same_rough(a, b):
    for k in ("n", "mean", "zmin", "zmax", "Sa", "Sq", "Sz"):
        assert a[k] == b[k] or (np.isnan(a[k]) and np.isnan(b[k])), k


def test_batch_equals_alone(env):
    import torch
    F, ctx, ws, alone = env
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    rough = torch.zeros(len(ws) * F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    ctx.predict_batch(tools, procs, outs, rough_buf=rough)
    torch.cuda.synchronize()
    rs = rough_array(F, rough, len(ws))
    for (ref, rref), out, r in zip(alone, outs, rs):
        assert torch.equal(out, ref)
        same_rough(r, rref)


def test_prepared_batch_graph_replay(env):
    import torch
    F, ctx, ws, alone = env
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    rough = torch.zeros(len(ws) * F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    b = ctx.batch(tools, procs, outs, rough_buf=rough)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)  # warm run outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    for o in outs:
        o.fill_(123.0)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    rs = rough_array(F, rough, len(ws))
    for (ref, rref), out, r in zip(alone, outs, rs):
        assert torch.equal(out, ref)
        same_rough(r, rref)


def test_batch_against_oracle(env, oracle_mod):
    F, ctx, ws, alone = env
    for w, (out, _) in list(zip(ws, alone))[:6]:
        ref = oracle_mod.fsm(W.Workload(w.name, w.tool, w.process.replace(precision="fp64")), n_threads=8)
        compare_maps(out, ref, w.process.precision)


def test_server_results_equal_alone_and_in_the_mix(env):
    import torch
    F, ctx, ws, alone = env
    ctx.server_start(budget_bytes=256 << 20, n_streams=3, max_batch=5)
    try:
        handles = [(ctx.tool(w.tool), ctx.process(w.process)) for w in ws]
        rng = np.random.default_rng(5)
        tickets = []
        for t, p in handles:  # staggered arrivals while earlier batches run
            tickets.append(ctx.submit(t, p))
            time.sleep(float(rng.exponential(0.002)))
        for tk, (ref, rref) in zip(tickets, alone):
            res = ctx.poll(tk, timeout_ms=60000)
            got = F.result_view(res)
            assert torch.equal(got, ref)
            same_rough(res["rough"], rref)
            assert res["latency_s"] >= res["queue_s"] >= 0.0
            ctx.release(tk)
    finally:
        ctx.server_stop()


def test_server_admission_budget(env):
    F, ctx, ws, alone = env
    big = W.raster_ball_d10(precision="fp64", width=1.0)  # 8 MB map
    ctx.server_start(budget_bytes=4 << 20, n_streams=1, max_batch=4)
    try:
        t, p = ctx.tool(big.tool), ctx.process(big.process)
        with pytest.raises(F.FsmError) as e:
            ctx.submit(t, p)
        assert e.value.status == -2
        # requests that fit one at a time are all served in order
        small = ws[:4]
        tickets = [ctx.submit(ctx.tool(w.tool), ctx.process(w.process)) for w in small]
        for tk, (ref, _) in zip(tickets, alone[:4]):
            res = ctx.poll(tk, timeout_ms=60000)
            import torch
            assert torch.equal(F.result_view(res), ref)
            ctx.release(tk)
    finally:
        ctx.server_stop()
