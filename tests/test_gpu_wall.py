"""Side-wall maps on the GPU: the same sweep over the map frame (x, z, -y) of
the wall the flank leaves on the +Y side of a pass, against the FP64 oracle
cell by cell at reduced sizes, and through size-independent properties on
the full 20 x 1 mm wall at 2 um (5 Mcells, 1.2e10 trajectory points)."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

from .gpu_common import SA_REL, compare_maps, compare_roughness, gpu_map

pytestmark = pytest.mark.gpu


def _wall_helix_runout_lead():
    tool = ToolSpec("flat", 4.0, 3, [35.0], n_edge=40, n_end=0, runout_mm=0.005, runout_phase_deg=20.0)
    proc = ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=3.0, ap=0.6, lead_deg=5.0, pass_x0=-0.6, pass_y0=0.0,
                       steps_per_pass=720, x0=-0.16, y0=-0.55, pitch=0.01, nx=32, ny=40, surface="wall",
                       wall_y=1.9)
    return Workload("wall_lead", tool, proc)


def _wall_climb_tilt():
    tool = ToolSpec("flat", 6.0, 4, [30.0, 32.0, 30.0, 32.0], n_edge=120, n_end=0, runout_mm=0.01,
                    runout_phase_deg=200.0)
    proc = ProcessSpec(fz=0.06, rpm=8000, rot_step_deg=0.5, ap=0.3, tilt_deg=3.0, rot_sense=-1,
                       pass_x0=-3.7, pass_y0=0.2, steps_per_pass=17000, x0=-0.301, y0=-0.2937, pitch=0.0023,
                       nx=257, ny=121, surface="wall", wall_y=3.0)
    return Workload("wall_climb", tool, proc)


CASES = {
    "side_wall_d12_reduced": lambda: W.side_wall_flat_d12(length=0.4, height=0.1),
    "wall_helix_runout_lead": _wall_helix_runout_lead,
    "wall_climb_tilt_ragged": _wall_climb_tilt,
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_wall_parity(oracle_mod, name, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w0 = CASES[name]()
    w = Workload(w0.name, w0.tool, w0.process.replace(precision=prec))
    ref = oracle_mod.fsm(w, n_threads=1)
    assert (ref.H < -w.process.wall_y).mean() > 0.2
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, ref, prec)
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == ref.stats["cutting"]
    else:
        assert abs(int(c[1]) - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2
    r = ctx.roughness(H)
    compare_roughness(r, oracle_mod.roughness(ref.H), SA_REL[prec])


def test_wall_trajectory(oracle_mod):
    """Trajectory records of a wall process are in its map frame (x, z, -y):
    the point of each edge deepest into the wall."""
    from paper_2603_28160_gb300 import fsm as F
    import torch
    w = _wall_helix_runout_lead()
    ctx = F.Context(0)
    raw = ctx.trajectory(ctx.tool(w.tool), ctx.process(w.process))
    torch.cuda.synchronize()
    xyz, j, _ = (a.cpu().numpy() for a in F.trajectory_views(raw, w.tool.n_teeth))
    xo, jo = oracle_mod.trajectory(w)
    assert np.abs(xyz[..., 2] - xo[..., 2]).max() <= 1e-9
    same = j == jo
    assert same.mean() > 0.999
    assert np.abs(xyz - xo)[same].max() <= 1e-9


def test_side_wall_full_size():
    """Full 20 x 1 mm wall: no cell beyond the stock or deeper than the tool
    reaches (radius plus runout), every cell cut, and FP32 within 5 nm of
    FP64 everywhere."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    maps = {}
    for prec in ("fp64", "fp32"):
        w = W.side_wall_flat_d12(precision=prec)
        H = gpu_map(ctx, F, w)
        stock = -w.process.wall_y
        deepest = -(w.process.pass_y0 + 0.5 * w.tool.diameter + w.tool.runout_mm)
        assert bool((H <= stock).all())
        # FP32 maps store heights as floats: 4.8e-7 mm ulp at 6 mm
        assert bool((H.double() >= deepest - (1e-9 if prec == "fp64" else 5e-6)).all())
        assert (H < stock).double().mean().item() == 1.0
        maps[prec] = H.double()
    d = (maps["fp32"] - maps["fp64"]).abs().max().item()
    assert d <= 5e-6, d
