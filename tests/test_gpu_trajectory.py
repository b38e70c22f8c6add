"""Trajectory maps on the GPU (Section 3.1: per time step, the lowest point of
every cutting edge and its global coordinates) against the FP64 oracle.

z is unique and compared everywhere (<= 1e-9 mm). The reported edge point is
the first of equal z; where rounding makes two points tie differently on the
two sides, the GPU's choice must be a valid one: the oracle's own pose of
that point lies within 1e-9 mm of the minimum, and the GPU's coordinates are
that pose."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _generic_ball():
    tool = ToolSpec("ball", 6.0, 3, [30.0, 33.0, 36.0], n_edge=25, runout_mm=0.006, runout_phase_deg=75.0)
    proc = ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=2.0, ap=0.2, pass_x0=-0.9, pass_y0=-0.05,
                       steps_per_pass=1080, n_passes=2, ae=0.05, x0=-0.1, y0=-0.1, pitch=0.01, nx=24, ny=24,
                       lead_deg=14.0, tilt_deg=-6.0)
    return Workload("ball_leaned", tool, proc)


def _flat_runout():
    tool = ToolSpec("flat", 4.0, 2, [30.0], n_edge=5, n_end=7, runout_mm=0.01, runout_phase_deg=40.0)
    proc = ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.5, pass_x0=-1.23, pass_y0=0.45,
                       steps_per_pass=900, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40, phase0_deg=3.0)
    return Workload("flat_runout", tool, proc)


CASES = {
    "ball_leaned": _generic_ball,
    "flat_runout_ties": _flat_runout,
    "slot_flat_d6": lambda: W.slot_flat_d6(),
    "insert_case2": lambda: W.paper_case(1, length=0.6, width=0.4, pitch=0.004, rot_step_deg=0.25, n_edge=61),
    "raster_ball_reduced": lambda: W.raster_ball_d10(precision="fp64", width=0.3, n_passes=2),
    # fed at 130 deg from +X, zig-zag: the path and tool turned about the start of pass 0
    "ball_leaned_fed_130": lambda: Workload("ball_fed_130", _generic_ball().tool,
                                            _generic_ball().process.replace(feed_dir_deg=130.0,
                                                                            pass_mode="zigzag")),
    "torus_zigzag": lambda: Workload("torus_zz", ToolSpec("torus", 4.0, 3, [30.0], n_edge=21, n_end=15,
                                                          corner_radius=0.7, runout_mm=0.003),
                                     ProcessSpec(fz=0.05, rpm=1000, rot_step_deg=1.0, ap=0.3, lead_deg=6.0,
                                                 pass_x0=-1.0, pass_y0=-0.1, steps_per_pass=700, n_passes=3,
                                                 ae=0.1, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40,
                                                 pass_mode="zigzag")),
}


def gpu_trajectory(w):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    raw = ctx.trajectory(t, p)
    torch.cuda.synchronize()
    xyz, j, K = F.trajectory_views(raw, w.tool.n_teeth)
    return raw, xyz.cpu().numpy(), j.cpu().numpy(), K.cpu().numpy()


def check(oracle_mod, w, xyz_g, j_g, K_g, s0=0):
    count = xyz_g.shape[0]
    xyz_o, j_o = oracle_mod.trajectory(w, s0=s0, count=count)
    assert (K_g == np.arange(w.tool.n_teeth)[None, :]).all()
    dz = np.abs(xyz_g[..., 2] - xyz_o[..., 2])
    assert dz.max() <= TOL, dz.max()
    same = j_g == j_o
    d = np.abs(xyz_g - xyz_o)[same]
    assert d.max() <= TOL, d.max()
    diff = np.argwhere(~same)
    assert len(diff) <= 1e-3 * j_g.size + 8, len(diff)
    for i, K in diff[:64]:
        pose = oracle_mod.pose(w, s0 + int(i), int(K), int(j_g[i, K]))
        assert abs(pose[2] - xyz_o[i, K, 2]) <= TOL
        assert np.abs(pose - xyz_g[i, K]).max() <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_trajectory_small(oracle_mod, name):
    w = CASES[name]()
    _, xyz, j, K = gpu_trajectory(w)
    assert xyz.shape[0] == w.process.n_passes * w.process.steps_per_pass
    check(oracle_mod, w, xyz, j, K)


def test_trajectory_independent_of_map_precision():
    a = gpu_trajectory(W.raster_ball_d10(precision="fp64", width=0.3, n_passes=2))[0]
    b = gpu_trajectory(W.raster_ball_d10(precision="fp32", width=0.3, n_passes=2))[0]
    assert bool((a == b).all())


def test_trajectory_fullsize_sampled(oracle_mod):
    """The 5 x 5 mm, 12-pass ball raster (every step of the tool path), with
    windows at the start, the middle and the end checked against the oracle."""
    w = W.raster_ball_d10(precision="fp32")
    _, xyz, j, K = gpu_trajectory(w)
    total = w.process.n_passes * w.process.steps_per_pass
    assert xyz.shape[0] == total
    for s0 in (0, total // 2 - 500, total - 1500):
        check(oracle_mod, w, xyz[s0:s0 + 1500], j[s0:s0 + 1500], K[s0:s0 + 1500], s0=s0)


def test_trajectory_rejects_short_buffer():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    w = _flat_runout()
    ctx = F.Context(0)
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    short = torch.empty((10, F.TRAJ_BYTES), dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FsmError):
        ctx.trajectory(t, p, out=short)
