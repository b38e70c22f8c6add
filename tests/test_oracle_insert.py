"""Pins of the oracle's round-insert face mill (Eq. eq_point_p_equation,
eq_tool_point_p_equation, eq_cutting_edge_to_tool): geometric invariants and
closed forms, not the oracle's own formulas."""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload


def insert_tool(**kw):
    base = dict(kind="insert", diameter=10.0, n_teeth=2, helix_deg=[0.0], n_edge=41, insert_radius=5.0)
    base.update(kw)
    return ToolSpec(**base)


def wl(tool, **kw):
    base = dict(fz=0.4, rpm=5400, rot_step_deg=0.5, ap=0.3, pass_x0=-12.0, pass_y0=0.0, steps_per_pass=100,
                x0=-0.3 + 0.31 * 0.005, y0=-0.3 + 0.37 * 0.005, pitch=0.005, nx=120, ny=120)
    base.update(kw)
    return Workload("insert", tool, ProcessSpec(**base))


def test_insert_edge_is_the_lower_circle_arc(oracle_mod):
    R, D, ap = 5.0, 10.0, 0.3
    w = wl(insert_tool(), ap=ap)
    q = oracle_mod.edge_points(w)[0]           # tooth 0, no rake, no runout
    assert np.allclose(q[:, 1], 0.0, atol=1e-15)
    centre = np.array([D / 2, 0.0, R])
    assert np.allclose(np.linalg.norm(q - centre, axis=1), R, atol=1e-12)
    assert (q[:, 2] <= R).all()                 # the lower semicircle
    dL = math.sqrt(R * R - (R - ap) ** 2)      # immersion branch of the discretisation length
    assert q[0, 0] - D / 2 == pytest.approx(-dL, abs=1e-12)
    assert q[-1, 0] - D / 2 == pytest.approx(dL, abs=1e-12)
    assert np.allclose(np.diff(q[:, 0]), 2 * dL / 40, atol=1e-12)


def test_insert_feed_branch_of_the_discretisation_length(oracle_mod):
    """Tiny depth: the half-length is set by the feed, fz / (2 cos gamma_f)."""
    gf = 3.0
    w = wl(insert_tool(rake_f_deg=gf), ap=0.001, fz=0.6)
    q0 = oracle_mod.edge_points(wl(insert_tool(), ap=0.001, fz=0.6))[0]
    half = 0.6 / (2 * math.cos(math.radians(gf)))
    q = oracle_mod.edge_points(w)[0]
    lowest = q[len(q) // 2]
    # arc length of the discretised edge from its lowest point to its end
    d = np.linalg.norm(q[-1] - lowest)
    assert np.linalg.norm(q0[-1] - q0[len(q0) // 2]) == pytest.approx(
        math.hypot(0.6 / 2, 5.0 - math.sqrt(25.0 - 0.09)), rel=1e-12)
    assert d == pytest.approx(math.hypot(half, 5.0 - math.sqrt(25.0 - half * half)), rel=1e-12)


def test_rake_is_a_rigid_rotation_about_the_lowest_point(oracle_mod):
    flat = oracle_mod.edge_points(wl(insert_tool()))[0]
    raked = oracle_mod.edge_points(wl(insert_tool(rake_f_deg=7.0, rake_p_deg=4.0)))[0]
    d0 = np.linalg.norm(flat[:, None] - flat[None], axis=2)
    d1 = np.linalg.norm(raked[:, None] - raked[None], axis=2)
    assert np.allclose(d0, d1, atol=1e-12)
    mid = len(flat) // 2
    assert np.allclose(raked[mid], [5.0, 0.0, 0.0], atol=1e-12)   # the lowest point does not move
    assert not np.allclose(raked, flat)


def test_per_insert_runout_moves_insert_k_by_k_eps(oracle_mod):
    er, ea = 0.011, 0.003          # Case 1 of the run-out table
    w = wl(insert_tool(n_teeth=3, eps_r_mm=er, eps_a_mm=ea))
    q = oracle_mod.edge_points(w)
    mid = q.shape[1] // 2
    for K in range(3):
        p = q[K, mid]
        ang = -2 * math.pi * K / 3
        r = 5.0 + K * er
        assert np.allclose(p, [r * math.cos(ang), r * math.sin(ang), K * ea], atol=1e-12)


def test_face_mill_depth_and_feed_periodicity(oracle_mod):
    """Zero runout: period fz; per-insert runout: period N fz; the lowest cut
    is at stock - ap."""
    for er, P_teeth in ((0.0, 1), (0.011, 2)):
        w = wl(insert_tool(eps_r_mm=er, eps_a_mm=0.003 if er else 0.0), fz=0.4, rot_step_deg=0.5,
               steps_per_pass=int(24.6 / (2 * 0.4 / 720)), pitch=0.005, nx=400, ny=60,
               x0=-1.0 + 0.31 * 0.005, y0=-0.15 + 0.37 * 0.005)
        r = oracle_mod.fsm(w, n_threads=1)
        assert r.H.min() == pytest.approx(-0.3, abs=1e-12)
        P = int(round(P_teeth * 0.4 / 0.005))
        ok = ~(r.flags[:, :-P] | r.flags[:, P:])
        assert np.abs(r.H[:, :-P] - r.H[:, P:])[ok].max() <= 1e-9


def test_insert_gather_equals_scatter(oracle_mod):
    w = wl(insert_tool(rake_f_deg=0.6, eps_r_mm=-0.026, eps_a_mm=0.009), pass_x0=-1.0, steps_per_pass=3600,
           nx=24, ny=24, pitch=0.02, x0=4.6 + 0.31 * 0.02, y0=-0.24 + 0.37 * 0.02, rot_step_deg=0.25)
    r = oracle_mod.fsm(w)
    g = oracle_mod.gather(w, 1)
    assert r.stats["cutting"] > 500
    ok = ~r.flags
    assert np.array_equal(g[ok], r.H[ok])
