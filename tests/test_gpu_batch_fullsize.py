"""The full 4096-surface Latin-hypercube batch (about 5 Gcells) in the launch
configuration the benchmark times -- one prepared batch, replayed as a CUDA
graph -- with surfaces the oracle can afford checked cell by cell: the
cheapest ball-end and flat-end ones, chosen by trajectory-point count. Every
map of the batch is also checked against the stock bound and its roughness
record against the map it describes (n = cells, stock_z >= zmax)."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import compare_maps

pytestmark = pytest.mark.gpu


def test_full_batch_sampled_parity(oracle_mod):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    ws = W.lhs_batch(n=4096)
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    rough = torch.zeros(len(ws) * F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    b = ctx.batch(tools, procs, outs, rough_buf=rough)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b.run(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.run(s)
    for o in outs:
        o.fill_(123.0)
    g.replay()
    torch.cuda.synchronize()
    raw = rough.cpu().numpy().tobytes()
    sz = F.ROUGH_BYTES
    for i, (w, o) in enumerate(zip(ws, outs)):
        assert bool((o <= w.process.stock_z).all()), i
        r = F.rough_dict(F.RoughnessOut.from_buffer_copy(raw[i * sz:(i + 1) * sz]))
        assert r["n"] == w.process.cells and r["zmax"] <= w.process.stock_z
    balls = sorted((i for i, w in enumerate(ws) if w.tool.kind == "ball"), key=lambda i: ws[i].trajectory_points)
    flats = sorted((i for i, w in enumerate(ws) if w.tool.kind == "flat"), key=lambda i: ws[i].trajectory_points)
    for i in balls[:3] + flats[:1]:
        w = ws[i]
        ref = oracle_mod.fsm(W.Workload(w.name, w.tool, w.process.replace(precision="fp64")), n_threads=8)
        assert ref.stats["cutting"] > 0
        compare_maps(outs[i], ref, "fp32")
    b.close()
