"""A map larger than 2^31 cells (46341 x 46341 at 10 um, 8.6 GB in FP32):
the sweep, the store and the roughness reductions run past 32-bit cell
indices. A short pass of a ball end cuts a small region: that region equals
the oracle's map of a window placed on the same cells, every other cell keeps
the stock, and the roughness record describes all 2,147,488,281 cells."""
import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

from .gpu_common import compare_maps

pytestmark = pytest.mark.gpu

N = 46341                      # N * N > 2^31 - 1
PITCH = 0.01
X0 = -0.5 * N * PITCH + 0.31 * PITCH
Y0 = -0.5 * N * PITCH + 0.37 * PITCH


def process(nx, ny, x0, y0, precision):
    return ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=2.0, ap=0.2, pass_x0=-3.5, pass_y0=0.0, steps_per_pass=3000,
                       x0=x0, y0=y0, pitch=PITCH, nx=nx, ny=ny, precision=precision)


def test_map_beyond_32_bit_cell_indices(oracle_mod):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    assert N * N > 2 ** 31 - 1
    tool = ToolSpec("ball", 6.0, 2, [30.0], n_edge=60)
    w = Workload("max", tool, process(N, N, X0, Y0, "fp32"))
    ctx = F.Context(0)
    H = F.heights_tensor(w.process)
    ctx.predict_surface(ctx.tool(w.tool), ctx.process(w.process), H)
    torch.cuda.synchronize()
    # the window of cells the tool can reach: x in [-6.5, 6.5], y in [-2, 2]
    i0 = int(np.floor((-6.5 - X0) / PITCH))
    k0 = int(np.floor((-2.0 - Y0) / PITCH))
    ni, nk = 1300, 400
    win = Workload("win", tool, process(ni, nk, X0 + i0 * PITCH, Y0 + k0 * PITCH, "fp64"))
    ref = oracle_mod.fsm(win, n_threads=8)
    assert ref.stats["cutting"] > 1000
    Hw = H[k0:k0 + nk, i0:i0 + ni]
    compare_maps(Hw, ref, "fp32")
    cut_total = int((H < 0).sum().item())
    assert cut_total == int((Hw < 0).sum().item()) == int((ref.H < 0).sum())
    r = ctx.roughness(H)
    assert r["n"] == float(N) * N
    assert r["zmax"] == 0.0
    assert abs(r["zmin"] - ref.H.min()) <= 5e-6
    del H
    torch.cuda.empty_cache()
