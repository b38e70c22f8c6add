"""The autotuner picks a valid sweep configuration, records it, and the
tuned configuration computes the same surface (FP64: bit for bit; FP32:
within the FP32 tolerance of the oracle)."""
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import compare_maps

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_choice_computes_the_same_surface(oracle_mod, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w = W.raster_ball_d10(precision=prec, width=0.6, pitch=0.002, n_passes=5, n_edge=80, rot_step_deg=0.25)
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    base = F.heights_tensor(w.process)
    ctx.predict_surface(t, p, base, tile=(128, 64) if prec == "fp64" else (256, 48))
    out = F.heights_tensor(w.process)
    best = ctx.autotune(t, p, out, max_candidates=6)
    assert best["tile"][0] % 4 == 0 and best["tile"][1] >= 1 and best["sweep_ms"] > 0
    tuned = F.heights_tensor(w.process)
    ctx.predict_surface(t, p, tuned)  # no override: uses the recorded choice
    torch.cuda.synchronize()
    if prec == "fp64":
        assert torch.equal(tuned, base)
    ref = oracle_mod.fsm(W.Workload(w.name, w.tool, w.process.replace(precision="fp64")), n_threads=5)
    compare_maps(tuned, ref, prec)
