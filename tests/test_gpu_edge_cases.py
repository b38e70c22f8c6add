"""Degenerate and extreme inputs through the C ABI against the FP64 oracle:
single-cell and single-row grids, a patch the tool never reaches, a single
time step, the most teeth and fewest edge points allowed, a depth of cut
beyond the insert radius, reversed spindle sense with negative lead/tilt and
a raised stock, and descriptors the library must reject."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

from .gpu_common import compare_maps, gpu_map

pytestmark = pytest.mark.gpu


def proc(**kw):
    base = dict(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.3, pass_x0=-3.2, pass_y0=0.011, steps_per_pass=11000,
                x0=-0.05 + 0.31e-3, y0=-0.05 + 0.37e-3, pitch=0.002, nx=50, ny=50)
    base.update(kw)
    return ProcessSpec(**base)


BALL = ToolSpec("ball", 4.0, 2, [30.0], n_edge=40, runout_mm=0.003, runout_phase_deg=10.0)
FLAT = ToolSpec("flat", 4.0, 2, [30.0], n_edge=20, n_end=60)

CASES = {
    "one_cell": lambda: Workload("one_cell", BALL, proc(nx=1, ny=1, x0=-0.0007, y0=0.0103)),
    "one_row": lambda: Workload("one_row", FLAT, proc(nx=333, ny=1, x0=-0.3331, y0=0.0101)),
    "one_column": lambda: Workload("one_col", BALL, proc(nx=1, ny=257, x0=0.0013, y0=-0.2561)),
    "never_reached": lambda: Workload("far", BALL, proc(x0=40.0)),
    "single_step": lambda: Workload("one_step", FLAT, proc(steps_per_pass=1, pass_x0=0.0, x0=-2.05, y0=-2.05,
                                                          nx=2050, ny=2050, pitch=0.002)),
    "sixteen_teeth_two_points": lambda: Workload(
        "t16", ToolSpec("ball", 6.0, 16, [20.0], n_edge=2), proc(ap=0.5, steps_per_pass=1500, pass_x0=-4.0)),
    "insert_ap_beyond_radius": lambda: Workload(
        "deep", ToolSpec("insert", 4.0, 3, [0.0], n_edge=31, insert_radius=0.8, rake_f_deg=2.0, rake_p_deg=-1.0,
                         eps_r_mm=0.004, eps_a_mm=0.002),
        proc(ap=1.2, fz=0.05, pass_x0=-3.5, steps_per_pass=28000)),
    "reverse_sense_negative_lean_raised_stock": lambda: Workload(
        "rev", ToolSpec("flat", 3.0, 3, [25.0, 40.0, 32.0], n_edge=15, n_end=40, runout_mm=0.006),
        proc(rot_sense=-1, phase0_deg=123.0, lead_deg=-6.0, tilt_deg=-9.0, stock_z=1.25, pass_x0=-3.0,
             steps_per_pass=13000, n_passes=3, ae=0.03)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_case_parity(oracle_mod, name, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w0 = CASES[name]()
    w = Workload(w0.name, w0.tool, w0.process.replace(precision=prec))
    ref = oracle_mod.fsm(w, n_threads=4)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, ref, prec)
    c = int(cnt[1].item())
    if prec == "fp64":
        assert c == ref.stats["cutting"]
    else:
        # FP32 counts a point by its FP32 cell near tile edges; all teeth of
        # a ball share the tip point, so such a point may count n_teeth times
        assert abs(c - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2 * w.tool.n_teeth
    if name == "never_reached":
        assert ref.stats["cutting"] == 0 and c == 0
        assert bool((H == w.process.stock_z).all())
    else:
        assert ref.stats["cutting"] > 0


def test_constant_map_roughness_is_flagged():
    """A map that is never cut is flat: Sa = Sq = Sz = 0 and Ssk, Sku NaN."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    H = torch.full((37, 41), -0.25, dtype=torch.float64, device="cuda")
    r = ctx.roughness(H)
    assert r["Sa"] == 0.0 and r["Sq"] == 0.0 and r["Sz"] == 0.0
    assert np.isnan(r["Ssk"]) and np.isnan(r["Sku"])


@pytest.mark.parametrize("bad", [
    dict(fz=0.0), dict(rot_step_deg=0.7), dict(rot_sense=2), dict(n_passes=0), dict(steps_per_pass=0),
    dict(nx=0), dict(pitch=-1.0), dict(lead_deg=89.5), dict(ap=float("nan")), dict(precision="fp16"),
])
def test_rejects_bad_process(bad):
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    with pytest.raises((F.FsmError, KeyError)):
        ctx.process(proc(**bad))


@pytest.mark.parametrize("tool", [
    ToolSpec("ball", 4.0, 17, [30.0], n_edge=5), ToolSpec("ball", 4.0, 2, [30.0], n_edge=1),
    ToolSpec("flat", 4.0, 2, [30.0], n_edge=5, n_end=1), ToolSpec("ball", -1.0, 2, [30.0], n_edge=5),
    ToolSpec("insert", 4.0, 2, [0.0], n_edge=5, insert_radius=0.0), ToolSpec("ball", 4.0, 2, [89.5], n_edge=5),
])
def test_rejects_bad_tool(tool):
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    with pytest.raises((F.FsmError, IndexError, ValueError)):
        ctx.tool(tool)


def test_pitch_below_the_fp32_guard_band(oracle_mod):
    """A 1 mm flat end at 1 nm pitch (a 2 x 2 um patch of 4 Mcells, crossed by
    the bottom edge as the tool turns): the FP32 error bound of the
    tile-local poses reaches a cell, more than the FP32 path's check of
    ambiguous points covers, so an FP32 map is refused; the FP64 map, whose
    ambiguous points are re-binned in FP64 from as many cells around the tile
    as the bound spans, equals the oracle cell by cell."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    tool = ToolSpec("flat", 1.0, 2, [30.0], n_edge=5, n_end=200)
    fine = dict(fz=0.001, rot_step_deg=0.1, ap=0.1, pitch=1e-6, nx=2000, ny=2000, x0=0.0, y0=0.0,
                pass_x0=-0.2, pass_y0=0.001, steps_per_pass=20000)
    w32 = Workload("fine32", tool, proc(precision="fp32", **fine))
    with pytest.raises(F.FsmError):
        ctx.predict_surface(ctx.tool(w32.tool), ctx.process(w32.process), F.heights_tensor(w32.process))
    w64 = Workload("fine64", tool, proc(precision="fp64", **fine))
    ref = oracle_mod.fsm(w64, n_threads=8)
    assert ref.stats["cutting"] > 0
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w64, counters=cnt)
    compare_maps(H, ref, "fp64")
    assert int(cnt[1].item()) == ref.stats["cutting"]
