"""Pins of the FP64 CPU oracle against closed forms, invariants, library
routines and brute force -- nothing here re-types the oracle's own formulas.

Paper references: kinematic chain Eq. eq_full_transformation (Section 2.1),
discretisation Section 2.2, sampling boundaries Eq. eq_sampling_boundaries and
the per-cell minimum (Section 2.3), roughness indicators Section 4.1.2.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

pytestmark = []


def wl(tool, **kw):
    base = dict(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.5, pass_x0=-1.23, pass_y0=0.45,
                steps_per_pass=100, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40)
    base.update(kw)
    return Workload("pin", tool, ProcessSpec(**base))


def Rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


# --------------------------------------------------------------------------
# Kinematic chain (Eq. eq_tool_to_spindle, eq_spindle_to_workpiece,
# eq_full_transformation): hand-derived trochoids.
# --------------------------------------------------------------------------
def test_pose_trochoid_flat_end(oracle_mod):
    tool = ToolSpec("flat", 4.0, 2, [0.0], n_edge=3, n_end=5)
    w = wl(tool, phase0_deg=10.0, n_passes=2, ae=0.2)
    p = w.process
    fs = 2 * 0.1 / 360.0
    for s in (0, 1, 7, 150, 199):
        pas, n = divmod(s, p.steps_per_pass)
        theta = math.radians(10.0 + (s % 360) * 1.0)
        for K in (0, 1):
            for j in range(5):            # bottom-edge points, r = 2 j / 4
                r = 2.0 * j / 4
                a = theta - math.pi * K   # tooth K sits 180 deg behind tooth 0
                exp = [p.pass_x0 + n * fs + r * math.cos(a), p.pass_y0 + pas * p.ae + r * math.sin(a),
                       -0.5]
                got = oracle_mod.pose(w, s, K, j)
                assert np.allclose(got, exp, atol=1e-13), (s, K, j, got, exp)


@pytest.mark.parametrize("sense", [1, -1])
def test_pose_helix_runout_sense(oracle_mod, sense):
    R, beta, rho, lam = 3.0, 30.0, 0.01, 40.0
    tool = ToolSpec("flat", 2 * R, 3, [beta], n_edge=5, n_end=0, runout_mm=rho,
                    runout_phase_deg=lam)
    w = wl(tool, ap=0.8, rot_sense=sense, phase0_deg=5.0)
    p = w.process
    fs = 3 * 0.1 / 360.0
    for s in (0, 3, 91):
        theta = math.radians(5.0 + sense * (s % 360))
        for K in range(3):
            for j in range(5):            # flank points, h = 0.8 j / 4
                h = 0.8 * j / 4
                alpha = -math.radians(120.0 * K) - sense * h * math.tan(math.radians(beta)) / R
                q = np.array([R * math.cos(alpha) + rho * math.cos(math.radians(lam)),
                              R * math.sin(alpha) + rho * math.sin(math.radians(lam)), h])
                exp = np.array([p.pass_x0 + s * fs, p.pass_y0, -0.8]) + Rz(theta) @ q
                assert np.allclose(oracle_mod.pose(w, s, K, j), exp, atol=1e-13)


def test_pose_lead_tilt_against_scipy(oracle_mod):
    L, T = 12.0, -7.0
    tool = ToolSpec("ball", 8.0, 2, [25.0], n_edge=7, runout_mm=0.004, runout_phase_deg=200.0)
    w = wl(tool, lead_deg=L, tilt_deg=T, ap=0.3)
    A = (Rotation.from_rotvec([-math.radians(T), 0, 0]) *
         Rotation.from_rotvec([0, math.radians(L), 0])).as_matrix()
    # stated convention: lead leans the axis toward +X, tilt toward +Y
    axis = A @ np.array([0.0, 0.0, 1.0])
    Lr, Tr = math.radians(L), math.radians(T)
    assert np.allclose(axis, [math.sin(Lr), math.sin(Tr) * math.cos(Lr), math.cos(Tr) * math.cos(Lr)])
    q = oracle_mod.edge_points(w)
    zr = oracle_mod.z_ref(w)
    p = w.process
    fs = 2 * 0.1 / 360.0
    for s in (0, 33, 77):
        theta = math.radians(s % 360)
        c = np.array([p.pass_x0 + s * fs, p.pass_y0, zr])
        for K in range(2):
            for j in range(7):
                exp = c + A @ Rz(theta) @ q[K, j]
                assert np.allclose(oracle_mod.pose(w, s, K, j), exp, atol=1e-12)


# --------------------------------------------------------------------------
# Edge discretisation (Section 2.2, generalised to end mills)
# --------------------------------------------------------------------------
def test_ball_profile_on_sphere_and_cap(oracle_mod):
    R, ap, L, T = 5.0, 0.2, 15.0, 4.0
    tool = ToolSpec("ball", 2 * R, 1, [0.0], n_edge=11)
    w = wl(tool, ap=ap, lead_deg=L, tilt_deg=T)
    q = oracle_mod.edge_points(w)[0]
    r, h = q[:, 0], q[:, 2]
    assert np.allclose(q[:, 1], 0.0, atol=1e-15)
    assert np.allclose(r ** 2 + (R - h) ** 2, R ** 2, atol=1e-12)
    kappa = np.arctan2(r, R - h)
    tau = math.acos(math.cos(math.radians(L)) * math.cos(math.radians(T)))
    half = math.acos((R - ap) / R)
    assert kappa[0] == pytest.approx(max(0.0, tau - half), abs=1e-12)
    assert kappa[-1] == pytest.approx(min(math.pi / 2, tau + half), abs=1e-12)
    assert np.allclose(np.diff(kappa), (kappa[-1] - kappa[0]) / 10, atol=1e-12)


def test_flat_profile_layout(oracle_mod):
    tool = ToolSpec("flat", 6.0, 1, [0.0], n_edge=4, n_end=7)
    w = wl(tool, ap=0.9)
    q = oracle_mod.edge_points(w)[0]
    assert np.allclose(q[:7, 0], np.linspace(0, 3.0, 7)) and np.allclose(q[:7, 2], 0)
    assert np.allclose(q[7:, 0], 3.0) and np.allclose(q[7:, 2], np.linspace(0, 0.9, 4))


def test_z_ref_puts_lowest_point_at_depth(oracle_mod):
    """Sweep every edge point through a dense revolution: the lowest z reached
    is stock - ap, and nothing goes lower."""
    tool = ToolSpec("ball", 10.0, 3, [30.0], n_edge=40, runout_mm=0.01, runout_phase_deg=70.0)
    w = wl(tool, ap=0.2, lead_deg=9.0, tilt_deg=6.0, stock_z=0.3)
    A = (Rotation.from_rotvec([-math.radians(6.0), 0, 0]) *
         Rotation.from_rotvec([0, math.radians(9.0), 0])).as_matrix()
    q = oracle_mod.edge_points(w).reshape(-1, 3)
    th = np.linspace(0, 2 * np.pi, 20001)
    z = oracle_mod.z_ref(w) + np.einsum("k,tkj,nj->nt", A[2], np.stack([
        np.stack([np.cos(th), -np.sin(th), 0 * th], -1),
        np.stack([np.sin(th), np.cos(th), 0 * th], -1),
        np.stack([0 * th, 0 * th, 1 + 0 * th], -1)], 1), q)
    assert z.min() >= 0.3 - 0.2 - 1e-12
    assert z.min() == pytest.approx(0.3 - 0.2, abs=1e-9)


# --------------------------------------------------------------------------
# Per-cell minimum invariants (Section 2.3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["flat", "ball"])
def test_stock_bound(oracle_mod, kind):
    tool = ToolSpec(kind, 4.0, 3, [20.0, 30.0, 40.0], n_edge=30, n_end=20 if kind == "flat" else 0,
                    runout_mm=0.006, runout_phase_deg=11.0)
    w = wl(tool, fz=0.05, ap=0.15, lead_deg=7.0, tilt_deg=3.0, pass_x0=-2.5, pass_y0=0.0,
           steps_per_pass=12000, n_passes=2, ae=0.1, stock_z=0.25)
    r = oracle_mod.fsm(w)
    assert (r.H <= 0.25).all()
    assert r.H.min() >= 0.25 - 0.15 - 1e-12
    assert r.stats["cutting"] > 0


def test_flat_floor_is_exact_depth(oracle_mod):
    from paper_2603_28160_gb300.workloads import slot_flat_d6
    w = slot_flat_d6()
    r = oracle_mod.fsm(w)
    assert r.stats["cells_hit"] == w.process.cells
    assert (r.H == w.process.stock_z - w.process.ap).all()


def test_flat_floor_with_runout_is_exact_depth(oracle_mod):
    tool = ToolSpec("flat", 2.0, 2, [30.0], n_edge=10, n_end=400, runout_mm=0.01,
                    runout_phase_deg=45.0)
    w = wl(tool, fz=0.05, ap=0.3, pass_x0=-1.3, pass_y0=0.0, steps_per_pass=9000)
    r = oracle_mod.fsm(w)
    cut = r.H < 0.0
    assert cut.sum() > 0.5 * r.H.size
    assert (r.H[cut] == -0.3).all()


def test_vertical_ball_tip_drags_the_pass_line(oracle_mod):
    """Without runout or lead the ball tip sits on the spindle axis, so it cuts
    the pass centre-line at full depth at every step."""
    tool = ToolSpec("ball", 6.0, 2, [30.0], n_edge=30)
    w = wl(tool, fz=0.1, ap=0.1, pass_x0=-1.5, pass_y0=0.0, steps_per_pass=6000,
           x0=-0.1 + 0.3 * 0.005, y0=-0.1 + 0.37 * 0.005)
    r = oracle_mod.fsm(w)
    row = int(math.floor((0.0 - w.process.y0) / w.process.pitch))
    assert (r.H[row] == -0.1).all()


def _scallop(R, d):
    return R - math.sqrt(R * R - d * d)


@pytest.mark.parametrize("n_teeth", [2, 3])
def test_feed_scallop_on_centre_line_leaned_ball(oracle_mod, n_teeth):
    """Lead larger than the engagement half-angle: the tip no longer touches,
    each tooth crossing of the centre-line leaves a circle of radius R, one per
    feed per tooth, so the centre-line scallop is R - sqrt(R^2 - (fz/2)^2)."""
    R, fz, ap, lead, pitch = 5.0, 0.2, 0.02, 20.0, 0.001
    tool = ToolSpec("ball", 2 * R, n_teeth, [0.0], n_edge=1200)
    S = 12000
    fs = n_teeth * fz / S
    xoff = R * math.sin(math.radians(lead))
    W = 0.8
    x0 = 0.3183 * pitch
    start = x0 - xoff - 0.5
    steps = int((W + 1.0) / fs)
    w = wl(tool, fz=fz, rot_step_deg=360.0 / S, ap=ap, lead_deg=lead, pass_x0=start, pass_y0=0.0,
           steps_per_pass=steps, x0=x0, y0=-3.3678 * pitch, pitch=pitch, nx=int(W / pitch), ny=7)
    r = oracle_mod.fsm(w)
    row = 3
    prof = r.H[row, 20:-20]
    assert prof.min() == pytest.approx(-ap, abs=2e-6)
    assert prof.max() - prof.min() == pytest.approx(_scallop(R, fz / 2), rel=0.03)


def test_stepover_scallop_mid_line(oracle_mod):
    """Two passes of a vertical ball, fz << ae: midway between the passes the
    lowest height is the trough cusp R - sqrt(R^2 - (ae/2)^2) above the floor."""
    R, fz, ae, ap, pitch = 5.0, 0.05, 0.4, 0.05, 0.001
    tool = ToolSpec("ball", 2 * R, 2, [0.0], n_edge=400)
    S = 1800
    fs = 2 * fz / S
    W = 0.3
    x0 = 0.3183 * pitch
    steps = int((W + 1.6) / fs)
    mid = 0.2
    w = wl(tool, fz=fz, rot_step_deg=360.0 / S, ap=ap, pass_x0=x0 - 0.8, pass_y0=0.0,
           steps_per_pass=steps, n_passes=2, ae=ae, x0=x0, y0=mid - 2.5 * pitch, pitch=pitch,
           nx=int(W / pitch), ny=5)
    r = oracle_mod.fsm(w)
    line = r.H[2, 10:-10]
    assert line.min() == pytest.approx(-ap + _scallop(R, ae / 2), rel=0.0, abs=0.05 * _scallop(R, ae / 2))


@pytest.mark.parametrize("runout", [0.0, 0.005])
def test_feed_periodicity(oracle_mod, runout):
    """S/N integer and fz/pitch integer: the map repeats every fz along the
    feed without runout, every N fz with runout."""
    N, fz, pitch = 4, 0.02, 0.002
    tool = ToolSpec("ball", 3.0, N, [30.0], n_edge=60, runout_mm=runout, runout_phase_deg=30.0)
    w = wl(tool, fz=fz, rot_step_deg=0.5, ap=0.05, lead_deg=0.0, pass_x0=-2.1, pass_y0=0.0,
           steps_per_pass=int(4.6 / (N * fz / 720)), x0=-0.2 + 0.31 * pitch, y0=-0.1 + 0.37 * pitch,
           pitch=pitch, nx=200, ny=100)
    r = oracle_mod.fsm(w)
    P = int(round((N * fz if runout else fz) / pitch))
    a, b = r.H[:, :-P], r.H[:, P:]
    ok = ~(r.flags[:, :-P] | r.flags[:, P:])
    assert ok.mean() > 0.999
    assert np.abs(a - b)[ok].max() <= 1e-9
    if runout:   # with runout the single-tooth period does not hold
        P1 = int(round(fz / pitch))
        assert np.abs(r.H[:, :-P1] - r.H[:, P1:]).max() > 1e-6


# --------------------------------------------------------------------------
# Brute-force inverse
# --------------------------------------------------------------------------
def _small_cases():
    ball = ToolSpec("ball", 4.0, 3, [30.0], n_edge=40, runout_mm=0.004, runout_phase_deg=30.0)
    flat = ToolSpec("flat", 3.0, 2, [35.0, 41.0], n_edge=12, n_end=60, runout_mm=0.006)
    return [
        wl(ball, fz=0.04, rot_step_deg=1.0, ap=0.1, lead_deg=10.0, pass_x0=-2.3, pass_y0=-0.05,
           steps_per_pass=9000, n_passes=3, ae=0.05, x0=-0.06 + 0.31 * 0.004,
           y0=-0.06 + 0.37 * 0.004, pitch=0.004, nx=30, ny=30),
        wl(flat, fz=0.05, rot_step_deg=2.0, ap=0.2, tilt_deg=3.0, pass_x0=-2.0, pass_y0=0.02,
           steps_per_pass=4000, x0=-0.05 + 0.31 * 0.005, y0=-0.05 + 0.37 * 0.005, pitch=0.005,
           nx=20, ny=20),
    ]


@pytest.mark.parametrize("case", [0, 1])
def test_gather_equals_scatter(oracle_mod, case):
    w = _small_cases()[case]
    r = oracle_mod.fsm(w)
    g = oracle_mod.gather(w, 1)
    assert r.stats["cutting"] > 1000
    ok = ~r.flags
    assert ok.mean() > 0.999
    assert np.array_equal(g[ok], r.H[ok])


def test_refined_gather_is_a_lower_bound_and_converges(oracle_mod):
    w = _small_cases()[0]
    r = oracle_mod.fsm(w)
    zr = r.stats["z_ref"]
    g2 = oracle_mod.gather(w, 2, z_ref=zr)
    g4 = oracle_mod.gather(w, 4, z_ref=zr)
    ok = ~r.flags
    assert (g2[ok] <= r.H[ok]).all() and (g4[ok] <= g2[ok]).all()
    gap1, gap2 = (r.H - g2)[ok].mean(), (g2 - g4)[ok].mean()
    assert gap1 > 0 and gap2 < gap1


# --------------------------------------------------------------------------
# Roughness (Section 4.1.2; ISO 25178-2 / ISO 4287 definitions)
# --------------------------------------------------------------------------
def test_roughness_sinusoid(oracle_mod):
    A, periods, nx, ny = 0.003, 7, 7 * 400, 9
    x = np.arange(nx)
    H = np.tile(A * np.sin(2 * np.pi * periods * x / nx), (ny, 1))
    r = oracle_mod.roughness(H)
    assert r["mean"] == pytest.approx(0.0, abs=1e-15)
    assert r["Sq"] == pytest.approx(A / math.sqrt(2), rel=1e-12)
    # discrete mean of |sin| over n samples per period: 2 cot(pi/n) / n (-> 2/pi)
    n = nx // periods
    sa = A * 2.0 / (n * math.tan(math.pi / n))
    assert r["Sa"] == pytest.approx(sa, rel=1e-12)
    assert sa == pytest.approx(2 * A / math.pi, rel=1e-4)
    assert r["Ssk"] == pytest.approx(0.0, abs=1e-9)
    assert r["Sku"] == pytest.approx(1.5, rel=1e-12)
    assert r["Sz"] == pytest.approx(2 * A, rel=1e-6)
    assert np.allclose(r["Ra_row"], sa, rtol=1e-12)


def test_roughness_two_level(oracle_mod):
    p, a = 0.2, 0.01          # fraction p of cells at height a, the rest at 0
    H = np.zeros((50, 100))
    H[:10, :] = a
    r = oracle_mod.roughness(H)
    mu = p * a
    sig = a * math.sqrt(p * (1 - p))
    assert r["mean"] == pytest.approx(mu, rel=1e-13)
    assert r["Sa"] == pytest.approx(2 * a * p * (1 - p), rel=1e-12)
    assert r["Sq"] == pytest.approx(sig, rel=1e-12)
    assert r["Ssk"] == pytest.approx((1 - 2 * p) / math.sqrt(p * (1 - p)), rel=1e-12)
    assert r["Sku"] == pytest.approx((1 - 3 * p * (1 - p)) / (p * (1 - p)), rel=1e-12)
    assert r["Sp"] == pytest.approx(a - mu) and r["Sv"] == pytest.approx(mu)


def test_roughness_random_vs_numpy(oracle_mod):
    rng = np.random.default_rng(1)
    H = rng.gamma(2.0, 0.001, size=(123, 77)) - 0.3
    r = oracle_mod.roughness(H, 10, 10)
    d = H - H.mean()
    assert r["Sa"] == pytest.approx(np.abs(d).mean(), rel=1e-12)
    assert r["Sq"] == pytest.approx(H.std(), rel=1e-12)
    assert r["Ssk"] == pytest.approx((d ** 3).mean() / H.std() ** 3, rel=1e-10)
    assert r["Sku"] == pytest.approx((d ** 4).mean() / H.std() ** 4, rel=1e-10)
    rows = [int((2 * k + 1) * 123 // 20) for k in range(10)]
    assert r["row_index"] == rows
    for k, row in enumerate(rows):
        prof = H[row]
        assert r["Ra_row"][k] == pytest.approx(np.abs(prof - prof.mean()).mean(), rel=1e-12)
        segs = np.array_split(np.arange(77), 5)
        # floor(q L / 5) boundaries: 15,15,15,15,17 for L = 77
        bounds = [(q * 77) // 5 for q in range(6)]
        rz = np.mean([np.ptp(prof[bounds[q]:bounds[q + 1]]) for q in range(5)])
        assert r["Rz_row"][k] == pytest.approx(rz, rel=1e-12)
        del segs


def test_roughness_sawtooth_profile(oracle_mod):
    """A row with one triangle per Rz segment of height 1 has Rz = 1."""
    L = 500
    t = np.arange(L)
    prof = np.abs(((t % 100) - 50) / 50.0)
    H = np.tile(prof, (5, 1))
    r = oracle_mod.roughness(H, 1, 0)
    assert r["Rz_row"][0] == pytest.approx(1.0, rel=1e-12)
    assert r["Ra_row"][0] == pytest.approx(np.abs(prof - prof.mean()).mean(), rel=1e-12)


# --------------------------------------------------------------------------
# Boundary ties (Eq. eq_sampling_boundaries is closed on both sides)
# --------------------------------------------------------------------------
def test_tie_flags_mark_both_cells(oracle_mod):
    """With the pass line exactly on a row boundary the vertical ball tip sits
    on that boundary at every step; both rows next to it are flagged."""
    tool = ToolSpec("ball", 4.0, 2, [0.0], n_edge=20)
    w = wl(tool, fz=0.1, ap=0.05, pass_x0=-2.5, pass_y0=0.0, steps_per_pass=9000, x0=-0.1,
           y0=-0.1, pitch=0.005, nx=40, ny=40)
    r = oracle_mod.fsm(w)
    assert r.flags[19].all() and r.flags[20].all()
    assert r.stats["cells_flagged"] >= 80
