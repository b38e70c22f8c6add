"""The paper's own Case 2 tool on the GPU: a face mill with two round inserts
(R = 5 mm, radial rake, per-insert radial/axial runout; Eq. eq_point_p_equation,
eq_tool_point_p_equation, eq_cutting_edge_to_tool). Every cell of the full
10 x 5 mm patch at 5 um pitch against the FP64 CPU oracle, for the three
conditions of the paper's Case 2 table, in FP64 and FP32."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import SA_REL, compare_maps, compare_roughness, gpu_map

pytestmark = pytest.mark.gpu

_REF = {}


def _reference(oracle_mod, i):
    if i not in _REF:
        _REF[i] = oracle_mod.fsm(W.paper_case(i, precision="fp64"), n_threads=1)
    return _REF[i]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("i", [0, 1, 2])
def test_paper_case2_insert(oracle_mod, i, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ref = _reference(oracle_mod, i)
    assert ref.stats["cutting"] > 0
    ctx = F.Context(0)
    w = W.paper_case(i, precision=prec)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, ref, prec)
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == ref.stats["cutting"]
    else:
        assert abs(int(c[1]) - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2
    r = ctx.roughness(H)
    ro = oracle_mod.roughness(ref.H)
    compare_roughness(r, ro, SA_REL[prec], keys=("Sa", "Sq"))


def test_paper_grid_batched(oracle_mod):
    """The nine cutting conditions of the paper's parameter grid, with the
    fixed 0.2 us time step of its performance table, as one batched FP32
    launch on 10 x 0.5 mm strips at 20 um (30 edge points), each map against
    the oracle."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    kw = dict(length=10.0, width=0.5, pitch=0.02, n_edge=30, dt_s=2e-7)
    ws = W.paper_grid(precision="fp32", **kw)
    refs = W.paper_grid(precision="fp64", **kw)
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    ctx.predict_batch(tools, procs, outs)
    torch.cuda.synchronize()
    for r, H in zip(refs, outs):
        ref = oracle_mod.fsm(r, n_threads=1)
        assert ref.stats["cutting"] > 0
        compare_maps(H, ref, "fp32")
