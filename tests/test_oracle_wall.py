"""Pins of the oracle's side-wall surface: the same edge points as the floor
map, sampled over (x, z) on the wall the flank leaves on the +Y side of a
pass, height -y (the wall's outward normal is -Y). Closed forms of
peripheral milling, not the oracle's own formulas."""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload


def wall(tool, **kw):
    base = dict(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=1.0, pass_x0=-1.5, pass_y0=0.0, steps_per_pass=5400,
                x0=-0.5, y0=-0.95, pitch=0.01, nx=100, ny=90, surface="wall", wall_y=2.5)
    base.update(kw)
    return Workload("wall", tool, ProcessSpec(**base))


def test_straight_flank_wall_rows_are_identical_and_reach_the_radius(oracle_mod):
    """Helix 0, vertical axis: every flank point of a tooth has the same x, y
    at a given step, so every wall row that a flank point reaches holds the
    same profile; the deepest point is the tool radius (a sample at 90 deg)."""
    R = 3.0
    w = wall(ToolSpec("flat", 2 * R, 2, [0.0], n_edge=201, n_end=0))
    r = oracle_mod.fsm(w)
    H = r.H
    assert r.stats["z_ref"] == -1.0
    hit = (H < -2.5).any(axis=1)
    assert hit.all()  # flank samples every 5 um, rows 10 um apart, all in [-1, 0]
    assert (H == H[0][None, :]).all()
    assert abs(H.min() + R) <= 1e-12
    assert (H >= -R - 1e-12).all()


def test_unreached_wall_cells_keep_the_stock(oracle_mod):
    """Rows below the tool tip and above the flank keep -wall_y exactly; rows
    holding a flank sample are cut across the whole patch (0.1 deg steps put
    samples 5 um apart along the 10 um cells)."""
    w = wall(ToolSpec("flat", 6.0, 2, [0.0], n_edge=11, n_end=0), ap=0.5, y0=-1.0, ny=120, pitch=0.01,
             rot_step_deg=0.1, steps_per_pass=54000)
    H = oracle_mod.fsm(w).H
    z = -1.0 + (np.arange(120) + 0.5) * 0.01
    assert (H[z < -0.5 - 0.01] == -2.5).all()
    assert (H[z > 0.0 + 0.01] == -2.5).all()
    sampled = np.unique(np.floor((-0.5 + 0.05 * np.arange(11) + 1.0) / 0.01).astype(int))
    sampled = sampled[sampled < 120]
    assert (H[sampled] < -2.5).all()
    others = np.setdiff1d(np.arange(120), sampled)
    assert (H[others] == -2.5).all()


def test_wall_is_the_binned_trochoid(oracle_mod):
    """One straight tooth: its flank point traces the trochoid
    (x_c + R cos theta, y_c + R sin theta) at fixed height; binning those
    closed-form points by x and keeping the largest y per cell gives the wall
    map (height -y)."""
    R, fz, dth = 5.0, 0.03, 0.05
    tool = ToolSpec("flat", 2 * R, 1, [0.0], n_edge=3, n_end=0)
    w = wall(tool, fz=fz, rot_step_deg=dth, ap=0.02, pass_x0=-0.25, steps_per_pass=7200 * 16, x0=-0.12,
             y0=-0.0125, pitch=0.005, nx=48, ny=1, wall_y=R - 0.2, phase0_deg=7.0)
    H = oracle_mod.fsm(w).H[0]
    s = np.arange(w.process.steps_per_pass)
    th = np.radians(7.0 + (s % 7200) * dth)
    x = -0.25 + s * (fz / 7200) + R * np.cos(th)
    y = R * np.sin(th)
    i = np.floor((x + 0.12) / 0.005).astype(int)
    keep = (i >= 0) & (i < 48) & (y > R - 0.2)
    exp = np.full(48, -(R - 0.2))
    np.minimum.at(exp, i[keep], -y[keep])
    assert (exp < -(R - 0.2)).all()
    assert np.abs(H - exp).max() <= 1e-12


def test_wall_feed_scallop(oracle_mod):
    """Peripheral milling with one tooth: the wall profile along the feed is
    the envelope of the edge's arcs, fz apart, and its peak-to-valley tends
    to R - sqrt(R^2 - (fz/2)^2). Here the trochoid adds a relative N fz /
    (pi R) = 0.5 % and the 1 um cells at most 2 pitch / fz = 0.7 %."""
    R, fz = 20.0, 0.3
    S = 600000
    tool = ToolSpec("flat", 2 * R, 1, [0.0], n_edge=3, n_end=0)
    w = wall(tool, fz=fz, rot_step_deg=360.0 / S, ap=0.02, pass_x0=-0.9, steps_per_pass=S * 6, x0=-0.45,
             y0=-0.0105, pitch=0.001, nx=900, ny=1, wall_y=R - 0.5)
    row = oracle_mod.fsm(w).H[0]
    assert (row < -(R - 0.5)).all()
    exact = R - math.sqrt(R * R - 0.25 * fz * fz)
    assert row.max() - row.min() == pytest.approx(exact, rel=0.02)
    assert row.min() == pytest.approx(-R, abs=1e-8)


def test_wall_gather_equals_scatter(oracle_mod):
    """Brute-force per-cell gather over the same samples, on the wall plane,
    with helix, runout and lead."""
    tool = ToolSpec("flat", 4.0, 3, [35.0], n_edge=40, n_end=0, runout_mm=0.005, runout_phase_deg=20.0)
    w = wall(tool, ap=0.6, lead_deg=5.0, rot_step_deg=3.0, steps_per_pass=720, pass_x0=-0.6, x0=-0.16,
             y0=-0.55, pitch=0.01, nx=32, ny=40, wall_y=1.9)
    r = oracle_mod.fsm(w)
    g = oracle_mod.gather(w)
    assert (r.H < -1.9).sum() > 100
    ok = ~r.flags
    assert np.array_equal(r.H[ok], g[ok])


def test_wall_needs_a_single_pass(oracle_mod):
    w = wall(ToolSpec("flat", 4.0, 2, [0.0], n_edge=5, n_end=0), n_passes=2, ae=0.1)
    with pytest.raises(ValueError):
        oracle_mod.fsm(w)
