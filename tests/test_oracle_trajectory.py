"""Pins of the oracle's trajectory map (Section 3.1: per time step, the lowest
point of every cutting edge and its global coordinates) against closed forms
and invariants that follow from the kinematic chain, not from the oracle."""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload


def wl(tool, **kw):
    base = dict(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.5, pass_x0=-1.23, pass_y0=0.45,
                steps_per_pass=400, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40)
    base.update(kw)
    return Workload("traj", tool, ProcessSpec(**base))


def test_vertical_ball_tip_is_the_trajectory(oracle_mod):
    """Ball end, no runout, vertical axis: the tip (edge point 0, on the axis)
    is the lowest point of every edge, at the tool reference position."""
    w = wl(ToolSpec("ball", 6.0, 3, [30.0], n_edge=9), n_passes=2, ae=0.25, ap=0.3)
    p = w.process
    xyz, j = oracle_mod.trajectory(w)
    assert xyz.shape == (800, 3, 3)
    assert (j == 0).all()
    fs = 3 * 0.1 / 360.0
    s = np.arange(800)
    pas, n = np.divmod(s, p.steps_per_pass)
    for K in range(3):
        assert np.allclose(xyz[:, K, 0], p.pass_x0 + n * fs, atol=1e-13)
        assert np.allclose(xyz[:, K, 1], p.pass_y0 + pas * p.ae, atol=1e-13)
        assert np.allclose(xyz[:, K, 2], -0.3, atol=1e-13)


def test_round_insert_traces_trochoids(oracle_mod):
    """Round inserts without rake or axis runout, odd point count: the middle
    point (the insert's lowest) of insert K runs on a trochoid of radius
    D/2 + K eps_r at height -ap + K eps_a, K tooth angles behind insert 0."""
    er, ea = 0.02, 0.004
    tool = ToolSpec("insert", 10.0, 2, [0.0], n_edge=11, insert_radius=5.0, eps_r_mm=er, eps_a_mm=ea)
    w = wl(tool, ap=0.4, phase0_deg=17.0, steps_per_pass=720)
    p = w.process
    xyz, j = oracle_mod.trajectory(w)
    assert (j == 5).all()
    fs = 2 * 0.1 / 360.0
    s = np.arange(720)
    theta = np.radians(17.0 + (s % 360))
    for K in range(2):
        r = 5.0 + K * er
        a = theta - math.pi * K
        assert np.allclose(xyz[:, K, 0], p.pass_x0 + s * fs + r * np.cos(a), atol=1e-12)
        assert np.allclose(xyz[:, K, 1], p.pass_y0 + r * np.sin(a), atol=1e-12)
        assert np.allclose(xyz[:, K, 2], -0.4 + K * ea, atol=1e-13)


def test_flat_end_tie_goes_to_the_first_point(oracle_mod):
    """Flat end, vertical axis: the whole bottom edge lies at the depth, a
    tie broken toward the first edge point (the axis); with axis runout that
    point circles the reference at radius rho, phase lambda ahead."""
    rho, lam = 0.01, 40.0
    tool = ToolSpec("flat", 4.0, 2, [30.0], n_edge=5, n_end=7, runout_mm=rho, runout_phase_deg=lam)
    w = wl(tool, phase0_deg=3.0)
    p = w.process
    xyz, j = oracle_mod.trajectory(w)
    assert (j == 0).all()
    s = np.arange(p.steps_per_pass)
    th = np.radians(3.0 + (s % 360) + lam)
    fs = 2 * 0.1 / 360.0
    for K in range(2):
        assert np.allclose(xyz[:, K, 0], p.pass_x0 + s * fs + rho * np.cos(th), atol=1e-13)
        assert np.allclose(xyz[:, K, 1], p.pass_y0 + rho * np.sin(th), atol=1e-13)
        assert (xyz[:, K, 2] == -0.5).all()


def _generic():
    tool = ToolSpec("ball", 6.0, 3, [30.0, 33.0, 36.0], n_edge=25, runout_mm=0.006, runout_phase_deg=75.0)
    return wl(tool, lead_deg=14.0, tilt_deg=-6.0, ap=0.2, rot_step_deg=2.0, steps_per_pass=1080, n_passes=2,
              ae=0.05, pass_x0=-0.9, pass_y0=-0.05, nx=24, ny=24, pitch=0.01)


def test_lowest_edge_point_depends_on_the_spindle_phase_only(oracle_mod):
    """The tool reference moves in a horizontal plane, so the argmin over an
    edge repeats every revolution: j(s) = j(s + S) and z(s) = z(s + S)."""
    w = _generic()
    S = 180
    xyz, j = oracle_mod.trajectory(w)
    assert (j[:-S] == j[S:]).all()
    assert np.array_equal(xyz[:-S, :, 2], xyz[S:, :, 2])
    assert len(np.unique(j)) > 1  # the lowest point moves along the leaned ball


def test_trajectory_is_the_minimum_over_the_edge(oracle_mod):
    """Brute force over single poses: z is the minimum over the edge points
    and the reported point is the first one attaining it."""
    w = _generic()
    xyz, j = oracle_mod.trajectory(w, s0=500, count=40)
    E = 25
    for i in range(0, 40, 7):
        s = 500 + i
        for K in range(3):
            z = np.array([oracle_mod.pose(w, s, K, jj)[2] for jj in range(E)])
            assert xyz[i, K, 2] == z.min() and j[i, K] == int(np.argmin(z))
            assert np.array_equal(xyz[i, K], oracle_mod.pose(w, s, K, int(j[i, K])))


def test_map_lies_below_every_landed_trajectory_point(oracle_mod):
    """The height map keeps the minimum over all points, so each cell is at
    or below the lowest edge points that landed in it."""
    w = _generic()
    p = w.process
    H = oracle_mod.fsm(w).H
    xyz, _ = oracle_mod.trajectory(w)
    pts = xyz.reshape(-1, 3)
    i = np.floor((pts[:, 0] - p.x0) / p.pitch).astype(int)
    k = np.floor((pts[:, 1] - p.y0) / p.pitch).astype(int)
    ok = (i >= 0) & (i < p.nx) & (k >= 0) & (k < p.ny) & (pts[:, 2] < 0)
    assert ok.sum() > 50
    assert (H[k[ok], i[ok]] <= pts[ok, 2]).all()


def test_rejects_out_of_range(oracle_mod):
    w = _generic()
    with pytest.raises(ValueError):
        oracle_mod.trajectory(w, s0=2000, count=200)
