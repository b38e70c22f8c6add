"""Surfaces fed off the X axis (feed_dir_deg, an extension: the paper feeds
along one axis, Eq. eq_spindle_to_workpiece) against the FP64 oracle.

A tilted feed turns the +X process's tool path and tool about the start of
pass 0; the grid stays axis-aligned. The sweep enumerates each point's steps
in the feed frame (the tile's extent along and across the feed) and bins in
the map frame, y stepping along the feed like x. Maps are compared cell by
cell with the oracle (Section 2.3's per-cell minimum over the points of Eq.
eq_sampling_boundaries) at several tiles with ragged edges, for both
precisions, both pass modes, a flat and a ball end and both phase-2 forms
(identical maps); batches that mix
tilted and +X surfaces must give every surface the map it gets alone, bit
for bit; the server the same.
"""
import math
import os

import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

from .gpu_common import SA_REL, compare_maps, gpu_map

pytestmark = pytest.mark.gpu


def _flat_fed(feed_dir):
    """A 3-flute flat end D3 (runout, unequal helix) on a 0.24 x 0.2 mm floor
    at 2 um, two overlapping passes fed at feed_dir."""
    pitch = 0.002
    tool = ToolSpec("flat", 3.0, 3, [35.0, 38.0, 41.0], n_edge=12, n_end=int(math.ceil(1.5 / (pitch / 2))),
                    runout_mm=0.006, runout_phase_deg=20.0)
    x0, y0, nx, ny = -0.12 + 0.31 * pitch, -0.1 + 0.37 * pitch, 120, 100
    px, py, spp = W.plan_passes_dir(tool, 0.05, 1.0, nx * pitch, ny * pitch, (0.0, 0.0), 2, 2.4, 0.3, pitch,
                                    feed_dir)
    return Workload("flat_fed", tool, ProcessSpec(fz=0.05, rpm=1000, rot_step_deg=1.0, ap=0.3, pass_x0=px,
                                                  pass_y0=py, steps_per_pass=spp, n_passes=2, ae=2.4, x0=x0,
                                                  y0=y0, pitch=pitch, nx=nx, ny=ny, feed_dir_deg=feed_dir))


CASES = {
    # the benchmark's tool at 30 deg, 0.3 mm square at 1 um (2 x 2 tiles, ragged)
    "ball_30": lambda: W.raster_ball_tilted(precision="fp64", width=0.3, feed_dir_deg=30.0, n_edge=60,
                                            rot_step_deg=0.5),
    # 200 deg, zig-zag: odd passes run back along the feed
    "ball_200_zigzag": lambda: W.raster_ball_tilted(precision="fp64", width=0.25, feed_dir_deg=200.0, n_edge=60,
                                                    rot_step_deg=0.5, pass_mode="zigzag"),
    # the direction (4, 3)/5 on a non-square patch, flat end with its bottom edge
    "flat_36.87": lambda: _flat_fed(math.degrees(math.atan2(3.0, 4.0))),
    # close to the Y axis
    "flat_95": lambda: _flat_fed(95.0),
}

_REF = {}


def reference(oracle_mod, name):
    if name not in _REF:
        _REF[name] = oracle_mod.fsm(CASES[name](), n_threads=os.cpu_count() or 1)
    return _REF[name]


@pytest.fixture(scope="module")
def F():
    from paper_2603_28160_gb300 import fsm
    return fsm


@pytest.fixture(scope="module")
def ctx(F):
    return F.Context(0)


def _with(w, **kw):
    return Workload(w.name, w.tool, w.process.replace(**kw))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tilted_feed_matches_oracle(ctx, F, oracle_mod, name, prec):
    import torch
    w = _with(CASES[name](), precision=prec)
    ref = reference(oracle_mod, name)
    assert ref.stats["cutting"] > 10000
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    tasks = torch.zeros(2, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt, form_tasks=tasks)
    compare_maps(H, ref, prec)
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == ref.stats["cutting"], (c, ref.stats)
    else:
        assert abs(int(c[1]) - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2
    t = tasks.cpu().numpy()
    assert t.sum() > 0
    # roughness of the tilted map
    r = ctx.roughness(H)
    o = oracle_mod.roughness(ref.H)
    for k in ("Sa", "Sq"):
        assert abs(r[k] - o[k]) <= SA_REL[prec] * abs(o[k]), (k, r[k], o[k])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_explicit_tiles(ctx, F, oracle_mod, prec):
    """Wide, short and small tiles: the tile's extent along and across the
    feed changes with its shape; the map must not."""
    w = _with(CASES["ball_30"](), precision=prec)
    ref = reference(oracle_mod, "ball_30")
    for tile in ((512, 24), (64, 64), (36, 100)):
        compare_maps(gpu_map(ctx, F, w, tile=tile), ref, prec)


def test_quarter_turn_permutes_the_gpu_map(ctx, F):
    """The process fed at 90 deg on the patch turned by 90 deg about the
    start of pass 0 gives the +X map with rows and columns permuted."""
    pitch = 0.004
    tool = ToolSpec("ball", 4.0, 3, [30.0], n_edge=40, runout_mm=0.004, runout_phase_deg=30.0)
    x0, y0 = -0.06 + 0.31 * pitch, -0.06 + 0.37 * pitch
    px, py = x0 - 600.5 * pitch, y0 + 10.5 * pitch
    base = ProcessSpec(fz=0.04, rpm=1000, rot_step_deg=1.0, ap=0.1, lead_deg=10.0, tilt_deg=3.0, pass_x0=px,
                       pass_y0=py, steps_per_pass=14760, n_passes=3, ae=0.02, x0=x0, y0=y0, pitch=pitch,
                       nx=30, ny=24)
    H0 = gpu_map(ctx, F, Workload("q0", tool, base)).cpu().numpy()
    Y1 = y0 + 24 * pitch
    turned = base.replace(feed_dir_deg=90.0, x0=px - (Y1 - py), y0=py + (x0 - px), nx=24, ny=30)
    H1 = gpu_map(ctx, F, Workload("q1", tool, turned)).cpu().numpy()
    want = H0.T[:, ::-1]
    assert H0.max() - H0.min() > 1e-3
    assert (np.abs(H1 - want) <= 1e-9).mean() > 0.99


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_mixing_tilted_and_axis_feeds(ctx, F, prec):
    """One batch launch per precision holds tilted and +X surfaces; each map
    equals the one predicted alone, bit for bit, and so does the server's."""
    import torch
    ws = [_with(CASES["ball_30"](), precision=prec),
          _with(W.raster_ball_d10(precision=prec, width=0.3, n_passes=2, n_edge=60, rot_step_deg=0.5)),
          _with(CASES["flat_95"](), precision=prec),
          _with(W.raster_ball_tilted(precision=prec, width=0.2, feed_dir_deg=-45.0, n_edge=40, rot_step_deg=1.0))]
    alone = [gpu_map(ctx, F, w) for w in ws]
    tools = [ctx.tool(w.tool) for w in ws]
    procs = [ctx.process(w.process) for w in ws]
    outs = [F.heights_tensor(w.process) for w in ws]
    ctx.predict_batch(tools, procs, outs)
    torch.cuda.synchronize()
    for a, b in zip(alone, outs):
        assert torch.equal(a, b)
    ctx.server_start(budget_bytes=1 << 30, n_streams=2, max_batch=4)
    try:
        tickets = [ctx.submit(t, p) for t, p in zip(tools, procs)]
        for tk, a in zip(tickets, alone):
            r = ctx.poll(tk, timeout_ms=60000)
            assert torch.equal(F.result_view(r), a)
            ctx.release(tk)
    finally:
        ctx.server_stop()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tilted_forms_match_oracle_and_each_other(ctx, F, oracle_mod, name, prec):
    """Each phase-2 form forced on a tilted feed: the item form (step windows
    from the turned tile's bounding box) and the phase form (revolution
    ranges of x and y against the tile itself) evaluate the same cutting
    points with the same arithmetic: the same map, bit for bit, and counts."""
    import torch
    w = _with(CASES[name](), precision=prec)
    ref = reference(oracle_mod, name)
    got = {}
    for form, slot in (("item", 0), ("phase", 1)):
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        tasks = torch.zeros(2, dtype=torch.int64, device="cuda")
        H = gpu_map(ctx, F, w, counters=cnt, form=form, form_tasks=tasks)
        compare_maps(H, ref, prec)
        t = tasks.cpu().numpy()
        assert t[slot] > 0 and t[1 - slot] == 0, (form, t)
        got[form] = (H.cpu().numpy(), cnt.cpu().numpy())
    assert np.array_equal(got["item"][0], got["phase"][0])
    assert got["item"][1][1] == got["phase"][1][1]  # cutting count
    assert got["phase"][1][0] <= got["item"][1][0]  # the phase form evaluates no more poses


def test_tilted_walls_are_rejected(ctx, F):
    wall = W.side_wall_flat_d12(precision="fp64", length=0.2)
    with pytest.raises(F.FsmError) as e:
        ctx.process(wall.process.replace(feed_dir_deg=20.0))
    assert e.value.status == -1
    # a whole turn is the +X feed itself
    ctx.process(wall.process.replace(feed_dir_deg=360.0))
