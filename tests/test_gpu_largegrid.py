"""The 20x20 mm, 2 um flat-end floor finish (100 Mcells, 3 flutes with
35/38/41 deg helix, runout 8 um) at full size. The oracle cannot cover 1.3e11
trajectory points in a test, so every cell is checked through properties that
hold at any size (element-by-element oracle parity of the same tool and
process runs at reduced size in test_gpu_parity.py):
  - no cell lies above the stock;
  - a vertical flat end cuts the floor at exactly stock - ap (bottom edge at
    h = 0), so every cut cell equals stock - ap exactly;
  - the FP32 map equals the FP64 map cell for cell (FP32 bins match FP64
    bins by the re-binning guard, and -ap is exact in both);
  - FP32 and FP64 count the same cutting evaluations to 1e-5: the FP32 path
    counts a point by its FP32 cell, so a point within FP32 error of a tile
    edge may be counted by both neighbouring tiles or by neither (its
    height still goes through the FP64 re-bin)."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_floor_finish_full_size():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    maps, counts = {}, {}
    for prec in ("fp32", "fp64"):
        w = W.floor_flat_d12(precision=prec)
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        H = F.heights_tensor(w.process)
        ctx.predict_surface(ctx.tool(w.tool), ctx.process(w.process), H, counters=cnt)
        torch.cuda.synchronize()
        stock, ap = w.process.stock_z, w.process.ap
        assert bool((H <= stock).all())
        cut = H < stock
        assert bool((H[cut] == stock - ap).all())
        assert cut.float().mean().item() > 0.99  # the floor is covered
        maps[prec] = H
        counts[prec] = cnt.cpu().numpy()
    diff = (maps["fp32"].double() != maps["fp64"]).double().mean().item()
    assert diff <= 1e-4, diff
    c32, c64 = counts["fp32"][1], counts["fp64"][1]
    assert abs(int(c32) - int(c64)) <= 1e-5 * c64 + 2
