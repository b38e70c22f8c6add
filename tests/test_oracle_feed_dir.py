"""Pins of the oracle's feed direction (an extension: the paper feeds along
one axis, Eq. eq_spindle_to_workpiece). A feed direction turns the whole
tool path and tool about the vertical through the start of pass 0, so:

- a quarter or half turn about a pivot on a cell centre maps the grid
  onto itself, and the map of the turned process on the turned patch is the
  0-degree map with its rows and columns permuted (exact up to boundary
  ties);
- at the direction (4, 3)/5, one feed per tooth is a whole number of cells
  along both axes, so the map repeats under that cell shift (the feed-mark
  periodicity of Section 2.3's per-cell minimum, in a direction that is not
  a grid axis).

A sign error in the turn, a path turned without the tool (or the tool
without the path) or a step-over on the wrong side fails one of these.
"""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

PITCH = 0.004


def _base(feed_dir=0.0, **kw):
    tool = ToolSpec("ball", 4.0, 3, [30.0], n_edge=40, runout_mm=0.004, runout_phase_deg=30.0)
    x0 = -0.06 + 0.31 * PITCH
    y0 = -0.06 + 0.37 * PITCH
    p = dict(fz=0.04, rpm=1000, rot_step_deg=1.0, ap=0.1, lead_deg=10.0, tilt_deg=3.0,
             pass_x0=x0 - 600.5 * PITCH, pass_y0=y0 + 10.5 * PITCH, steps_per_pass=14760, n_passes=3,
             ae=0.02, x0=x0, y0=y0, pitch=PITCH, nx=30, ny=24, feed_dir_deg=feed_dir)
    p.update(kw)
    return Workload("feed_dir_pin", tool, ProcessSpec(**p))


def _turned_patch(w, quarter):
    """The patch of w turned by quarter * 90 degrees about (pass_x0, pass_y0)."""
    p = w.process
    px, py, d = p.pass_x0, p.pass_y0, p.pitch
    X0, X1, Y0, Y1 = p.x0, p.x0 + p.nx * d, p.y0, p.y0 + p.ny * d
    if quarter == 1:    # (x, y) -> (px - (y - py), py + (x - px))
        return dict(x0=px - (Y1 - py), y0=py + (X0 - px), nx=p.ny, ny=p.nx)
    if quarter == 2:    # (x, y) -> (2 px - x, 2 py - y)
        return dict(x0=2 * px - X1, y0=2 * py - Y1, nx=p.nx, ny=p.ny)
    # quarter == 3:     (x, y) -> (px + (y - py), py - (x - px))
    return dict(x0=px + (Y0 - py), y0=py - (X1 - px), nx=p.ny, ny=p.nx)


def _permute(H, quarter):
    """Cell (i, k) of the 0-degree map seen on the turned patch."""
    if quarter == 1:
        return H.T[:, ::-1]
    if quarter == 2:
        return H[::-1, ::-1]
    return H.T[::-1, :]


@pytest.mark.parametrize("quarter", [1, 2, 3])
def test_quarter_turns_permute_the_map(oracle_mod, quarter):
    w0 = _base()
    r0 = oracle_mod.fsm(w0)
    assert r0.stats["cutting"] > 10000
    wq = _base(feed_dir=90.0 * quarter, **_turned_patch(w0, quarter))
    rq = oracle_mod.fsm(wq)
    want = _permute(r0.H, quarter)
    ok = ~(_permute(r0.flags, quarter) | rq.flags)
    assert ok.mean() > 0.99
    assert rq.stats["cutting"] == pytest.approx(r0.stats["cutting"], rel=1e-4)
    assert np.abs(rq.H - want)[ok].max() <= 1e-9
    # not vacuous: the map has relief, and the opposite quarter turn (or, for
    # the half turn, no turn) on the turned patch gives a different map
    assert r0.H.max() - r0.H.min() > 1e-3
    wrong_dir = {1: -90.0, 2: 0.0, 3: 90.0}[quarter]
    wrong = oracle_mod.fsm(_base(feed_dir=wrong_dir, **_turned_patch(w0, quarter)))
    assert np.abs(wrong.H - want)[ok].max() > 1e-4


@pytest.mark.parametrize("runout", [0.0, 0.005])
def test_periodicity_along_an_inclined_feed(oracle_mod, runout):
    """Feed direction (4, 3)/5, fz = 0.02 mm = (8, 6) cells of 2 um along
    (x, y): the map repeats under that shift without runout, under N times
    it with runout (and not under the single-tooth shift then)."""
    N, fz, pitch = 4, 0.02, 0.002
    theta = math.degrees(math.atan2(3.0, 4.0))
    c, s = 0.8, 0.6
    tool = ToolSpec("ball", 3.0, N, [30.0], n_edge=60, runout_mm=runout, runout_phase_deg=30.0)
    half = 1.9  # mm of path before and after the patch centre
    fs = N * fz / 720
    steps = int(2 * half / fs)
    cx, cy = 0.0123, -0.0077
    w = Workload("feed_dir_period", tool, ProcessSpec(
        fz=fz, rpm=1000, rot_step_deg=0.5, ap=0.05, pass_x0=cx - half * c, pass_y0=cy - half * s,
        steps_per_pass=steps, x0=cx - 0.2 + 0.31 * pitch, y0=cy - 0.1 + 0.37 * pitch, pitch=pitch,
        nx=200, ny=100, feed_dir_deg=theta))
    r = oracle_mod.fsm(w)
    assert (r.H < 0.0).mean() > 0.99  # the whole patch lies in the cut band
    k = N if runout else 1
    di, dk = 8 * k, 6 * k
    a, b = r.H[:-dk, :-di], r.H[dk:, di:]
    ok = ~(r.flags[:-dk, :-di] | r.flags[dk:, di:])
    assert ok.mean() > 0.999
    assert np.abs(a - b)[ok].max() <= 1e-9
    # the mirrored direction's shift does not repeat the map
    assert np.abs(r.H[dk:, :-di] - r.H[:-dk, di:]).max() > 1e-6
    if runout:
        assert np.abs(r.H[:-6, :-8] - r.H[6:, 8:]).max() > 1e-6


def test_zero_direction_is_the_axis_feed(oracle_mod):
    """feed_dir_deg = 0 and 360 give the same map (a full turn)."""
    w0 = _base()
    r0 = oracle_mod.fsm(w0)
    r1 = oracle_mod.fsm(_base(feed_dir=360.0))
    ok = ~(r0.flags | r1.flags)
    assert np.abs(r0.H - r1.H)[ok].max() <= 1e-9


def test_wall_rejects_a_feed_direction(oracle_mod):
    w = _base()
    wall = Workload("wall", w.tool, w.process.replace(surface="wall", n_passes=1, feed_dir_deg=10.0))
    with pytest.raises(Exception):
        oracle_mod.fsm(wall)
