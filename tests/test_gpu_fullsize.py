"""Full-size parity: the 5x5 mm, 1 um ball-end raster (25 Mcells, 12 passes)
in the launch configuration bench.py times, every cell against the FP64 CPU
oracle, in FP64 and FP32."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import SA_REL, compare_maps, compare_roughness, gpu_map

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def reference(oracle_mod):
    import os
    w = W.raster_ball_d10(precision="fp64")
    threads = min(os.cpu_count() or 1, w.process.n_passes)
    return oracle_mod.fsm(w, n_threads=threads)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fullsize_raster_ball(reference, oracle_mod, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w = W.raster_ball_d10(precision=prec)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, reference, prec)
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == reference.stats["cutting"]
    else:
        assert abs(int(c[1]) - reference.stats["cutting"]) <= 1e-5 * reference.stats["cutting"] + 2
    r = ctx.roughness(H)
    ro = oracle_mod.roughness(reference.H)
    compare_roughness(r, ro, SA_REL[prec], keys=("Sa", "Sq"))
    # stated tolerance on Ssk/Sku/Sz: same order as Sa/Sq relative to their scale
    for k in ("Sz", "Ssk", "Sku"):
        assert abs(r[k] - ro[k]) <= 10 * SA_REL[prec] * max(abs(ro[k]), 1.0), (k, r[k], ro[k])
