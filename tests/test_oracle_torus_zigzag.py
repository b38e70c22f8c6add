"""Pins of two extensions of the oracle: the bull-nose (torus) end mill and
zig-zag raster passes -- closed forms of their geometry, a reduction to the
ball end, exact floor depth, the bull-nose step-over cusp, and brute force."""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload


def wl(tool, **kw):
    base = dict(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.3, pass_x0=-1.23, pass_y0=0.45,
                steps_per_pass=100, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40)
    base.update(kw)
    return Workload("pin", tool, ProcessSpec(**base))


def profile(oracle_mod, w):
    pts = oracle_mod.edge_points(w)[0]       # tooth 0, no runout: r, h from x, y, z
    return np.hypot(pts[:, 0], pts[:, 1]), pts[:, 2]


@pytest.mark.parametrize("ap", [0.15, 0.3, 0.9])
def test_torus_profile_on_flat_arc_and_flank(oracle_mod, ap):
    """Bottom points on h = 0 inside R - rc, the rest on the corner arc
    (centre (R - rc, rc)) or the flank r = R, evenly spaced along the
    profile up to height ap."""
    R, rc = 2.0, 0.4
    w = wl(ToolSpec("torus", 2 * R, 2, [0.0], n_edge=41, n_end=9, corner_radius=rc), ap=ap)
    r, h = profile(oracle_mod, w)
    assert np.allclose(h[:9], 0.0) and np.allclose(r[:9], np.linspace(0, R - rc, 9), atol=1e-12)
    r, h = r[9:], h[9:]
    on_arc = h <= rc + 1e-12
    assert np.allclose((r[on_arc] - (R - rc)) ** 2 + (h[on_arc] - rc) ** 2, rc * rc, atol=1e-12)
    assert np.allclose(r[~on_arc], R, atol=1e-12)
    assert h[0] == 0.0 and abs(h[-1] - ap) < 1e-12
    # arc-length steps: chords on the arc, straight steps on the flank
    top = math.pi / 2 if ap >= rc else math.acos(1 - ap / rc)
    length = rc * top + max(0.0, ap - rc)
    ds = length / 40
    chord = np.hypot(np.diff(r), np.diff(h))
    both_arc = on_arc[1:] & on_arc[:-1]
    assert np.allclose(chord[both_arc], 2 * rc * math.sin(ds / (2 * rc)), atol=1e-12)
    both_flank = ~on_arc[1:] & ~on_arc[:-1]
    assert np.allclose(chord[both_flank], ds, atol=1e-12)


def test_torus_with_full_corner_is_the_ball(oracle_mod):
    """rc = D/2 without a bottom flat: the same points as the ball end
    (vertical axis: both are uniform in polar angle up to height ap)."""
    ball = wl(ToolSpec("ball", 5.0, 3, [25.0], n_edge=33), ap=0.7)
    tor = wl(ToolSpec("torus", 5.0, 3, [25.0], n_edge=33, n_end=0, corner_radius=2.5), ap=0.7)
    assert np.allclose(oracle_mod.edge_points(ball), oracle_mod.edge_points(tor), atol=1e-12)


def test_torus_floor_is_exact_depth(oracle_mod):
    """Vertical bull-nose: its bottom flat sits at stock - ap exactly. A flat
    end of diameter 2(R - rc) with the same bottom points samples the same
    positions, so every cell that tool's bottom reaches (exactly -ap there)
    is exactly -ap on the bull-nose map, and nothing is deeper."""
    tool = ToolSpec("torus", 3.0, 2, [30.0], n_edge=20, n_end=80, corner_radius=0.5)
    w = wl(tool, ap=0.25, rot_step_deg=2.0, pass_x0=-2.0, steps_per_pass=9000, pass_y0=0.0, x0=-0.1, y0=-0.1)
    H = oracle_mod.fsm(w).H
    flat = Workload("flat", ToolSpec("flat", 2.0, 2, [30.0], n_edge=2, n_end=80), w.process)
    Hf = oracle_mod.fsm(flat).H
    reached = Hf == -0.25
    assert reached.sum() > 200
    assert (H[reached] == -0.25).all()
    assert H.min() == -0.25


def test_torus_stepover_cusp(oracle_mod):
    """Two passes ae apart whose bottom flats do not meet: mid-way the corner
    arcs leave a cusp rc - sqrt(rc^2 - ((ae - 2(R - rc)) / 2)^2) above -ap
    (dense sampling: 0.1 deg steps, 2 um feed per revolution, 1.6 um along
    the profile)."""
    R, rc, ae = 1.0, 0.6, 1.3
    tool = ToolSpec("torus", 2 * R, 1, [0.0], n_edge=400, n_end=40, corner_radius=rc)
    w = wl(tool, ap=0.3, fz=0.002, rot_step_deg=0.1, pass_x0=-0.02, steps_per_pass=72000, n_passes=2, ae=ae,
           pass_y0=-0.5 * ae, x0=-0.02, y0=-0.01, pitch=0.002, nx=20, ny=10)
    H = oracle_mod.fsm(w, n_threads=2).H
    half = 0.5 * (ae - 2 * (R - rc))
    cusp = rc - math.sqrt(rc * rc - half * half)
    mid = H[4:6, :]                    # rows around y = 0, the mid-line
    assert (mid < 0).all()
    assert mid.max() + 0.3 == pytest.approx(cusp, rel=0.05)


def test_zigzag_odd_pass_runs_back(oracle_mod):
    """Zig-zag: step n of an odd pass sits where step spp-1-n of an even pass
    is, with the spindle still turning: the flat end's bottom points trace
    (x0 + (spp-1-n) fs + r cos(theta - phi_K), y_p + r sin(theta - phi_K))."""
    tool = ToolSpec("flat", 4.0, 2, [0.0], n_edge=3, n_end=5)
    w = wl(tool, phase0_deg=10.0, n_passes=3, ae=0.2, pass_mode="zigzag")
    p = w.process
    fs = 2 * 0.1 / 360.0
    for s in (0, 7, 100, 150, 199, 250):
        pas, n = divmod(s, p.steps_per_pass)
        theta = math.radians(10.0 + (s % 360))
        steps = (p.steps_per_pass - 1 - n) if pas % 2 else n
        for K in (0, 1):
            for j in range(5):
                r = 2.0 * j / 4
                a = theta - math.pi * K
                exp = [p.pass_x0 + steps * fs + r * math.cos(a), p.pass_y0 + pas * p.ae + r * math.sin(a), -0.3]
                assert np.allclose(oracle_mod.pose(w, s, K, j), exp, atol=1e-13), (s, K, j)


def test_zigzag_gather_equals_scatter(oracle_mod):
    tool = ToolSpec("ball", 3.0, 3, [35.0], n_edge=25, runout_mm=0.004, runout_phase_deg=50.0)
    w = wl(tool, ap=0.2, lead_deg=12.0, rot_step_deg=3.0, steps_per_pass=900, n_passes=3, ae=0.04,
           pass_x0=-2.0, pass_y0=-0.06, x0=-0.06, y0=-0.06, pitch=0.004, nx=30, ny=30, pass_mode="zigzag")
    r = oracle_mod.fsm(w)
    g = oracle_mod.gather(w)
    assert (r.H < 0).sum() > 200
    ok = ~r.flags
    assert np.array_equal(r.H[ok], g[ok])
    one = oracle_mod.fsm(Workload("oneway", tool, w.process.replace(pass_mode="one_way")))
    assert not np.array_equal(one.H, r.H)  # the return passes cut differently


def test_rejects_bad_torus_and_mode(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.fsm(wl(ToolSpec("torus", 2.0, 2, [0.0], n_edge=5, corner_radius=1.5)))
    with pytest.raises(ValueError):
        oracle_mod.fsm(wl(ToolSpec("torus", 2.0, 2, [0.0], n_edge=5, corner_radius=0.0)))
