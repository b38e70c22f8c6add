"""Seeded synthetic workloads: tool and process parameter sets.

This module only produces inputs -- tool geometry, cutting conditions, the
tool path (pass start points and step counts) and the sampling grid. It holds
none of the surface-generation arithmetic, so both the CUDA library and the
CPU oracle consume its output without sharing any computation.

The named workloads follow the configurations the surface generator is
measured on:

* ``slot_flat_d6``      flat end mill D=6, 2 flutes, one straight slot,
                        1x1 mm at 5 um (200x200 cells)
* ``raster_ball_d10``   ball end mill D=10, 4 flutes, runout 5 um, lead 15,
                        12 raster passes, 5x5 mm at 1 um (5000x5000 cells)
* ``floor_flat_d12``    flat end mill D=12, 3 flutes with 35/38/41 deg helix,
                        runout 8 um, 20x20 mm at 2 um (10000x10000 cells)
* ``lhs_batch``         Latin-hypercube batch of uneven patches
* ``poisson_stream``    request stream drawn from the batch distribution

Every patch origin is shifted from the pass centre-line by a generic
sub-cell amount (``CELL_OFFSET``) so that no systematic family of edge points
(the tool axis, a tooth crossing the centre-line) lies exactly on a sampling
boundary, where the paper's closed boundary intervals leave the cell ambiguous.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

MAX_TEETH = 16
# generic sub-cell offsets of the patch origin relative to the pass centre-line
CELL_OFFSET = (0.318309886183791, 0.367879441171442)


@dataclass
class ToolSpec:
    kind: str                     # "flat", "ball", "insert" (round inserts) or "torus" (bull-nose)
    diameter: float               # mm (inserts: radius of the inserts' lowest points x 2)
    n_teeth: int
    helix_deg: List[float]        # one per tooth
    tooth_deg: Optional[List[float]] = None  # angular positions; None = even pitch
    runout_mm: float = 0.0        # spindle-axis offset, rotates with the tool
    runout_phase_deg: float = 0.0
    n_edge: int = 50              # flank (flat) / meridian (ball) / corner + flank (torus) points
    n_end: int = 0                # flat / torus bottom-edge points (0 or >= 2)
    insert_radius: float = 0.0    # round insert radius R
    rake_f_deg: float = 0.0       # radial rake (gamma_f)
    rake_p_deg: float = 0.0       # axial rake (gamma_p)
    eps_r_mm: float = 0.0         # insert K sits K * eps_r further out ...
    eps_a_mm: float = 0.0         # ... and K * eps_a higher
    corner_radius: float = 0.0    # torus: corner radius rc, 0 < rc <= D/2

    def teeth_angles(self) -> List[float]:
        if self.tooth_deg is not None:
            return list(self.tooth_deg)
        return [360.0 * k / self.n_teeth for k in range(self.n_teeth)]

    def helix(self) -> List[float]:
        h = list(self.helix_deg)
        if len(h) == 1:
            h = h * self.n_teeth
        return h


@dataclass
class ProcessSpec:
    fz: float                     # feed per tooth, mm
    rpm: float
    rot_step_deg: float           # spindle angle per time step
    ap: float                     # axial depth of cut, mm
    pass_x0: float                # tool reference x at the first step of each pass
    pass_y0: float                # y of pass 0
    steps_per_pass: int
    x0: float                     # grid origin (corner of cell 0,0)
    y0: float
    pitch: float                  # sampling interval
    nx: int
    ny: int
    n_passes: int = 1
    ae: float = 0.0               # step-over, +Y
    phase0_deg: float = 0.0
    rot_sense: int = 1
    lead_deg: float = 0.0
    tilt_deg: float = 0.0
    stock_z: float = 0.0
    precision: str = "fp64"       # "fp64" or "fp32"
    surface: str = "floor"        # "floor" (grid x, y; height z) or "wall" (+Y side wall:
    wall_y: float = 0.0           # grid x, z; height -y; un-machined at y = wall_y)
    pass_mode: str = "one_way"    # "one_way" or "zigzag" (odd passes run back along -X)
    feed_dir_deg: float = 0.0     # feed direction: the path and tool turned about (pass_x0, pass_y0)

    def replace(self, **kw) -> "ProcessSpec":
        return dataclasses.replace(self, **kw)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    @property
    def trajectory_steps(self) -> int:
        return self.n_passes * self.steps_per_pass


@dataclass
class Workload:
    name: str
    tool: ToolSpec
    process: ProcessSpec
    note: str = ""

    @property
    def trajectory_points(self) -> int:
        """Every (time step, tooth, edge point) triple of the tool path."""
        per_tooth = self.tool.n_edge + (self.tool.n_end if self.tool.kind in ("flat", "torus") else 0)
        return self.process.trajectory_steps * self.tool.n_teeth * per_tooth


def plan_passes(tool: ToolSpec, fz: float, rot_step_deg: float, width: float,
                centre_x: float, first_y: float, ap: float, pitch: float):
    """Tool path: straight passes along +X, centred on the patch, long enough
    that the whole tool (radius D/2 plus runout plus depth) clears the patch at
    both ends. Returns (pass_x0, pass_y0, steps_per_pass)."""
    steps_per_rev = int(round(360.0 / rot_step_deg))
    feed_per_step = tool.n_teeth * fz / steps_per_rev
    overtravel = 0.5 * tool.diameter + tool.runout_mm + ap + 2.0 * pitch + tool.insert_radius
    half_steps = int(math.ceil((0.5 * width + overtravel) / feed_per_step))
    pass_x0 = centre_x - half_steps * feed_per_step
    return pass_x0, first_y, 2 * half_steps + 1


def _patch(width_x: float, width_y: float, pitch: float, centre=(0.0, 0.0)):
    nx = int(round(width_x / pitch))
    ny = int(round(width_y / pitch))
    x0 = centre[0] - 0.5 * nx * pitch + CELL_OFFSET[0] * pitch
    y0 = centre[1] - 0.5 * ny * pitch + CELL_OFFSET[1] * pitch
    return x0, y0, nx, ny


def slot_flat_d6(precision: str = "fp64") -> Workload:
    """Flat end mill D=6 mm, 2 flutes, helix 30 deg, no runout, one straight
    slot at fz=0.1 mm/tooth, 1000 rpm, ap=1 mm in 50 axial points, 0.5 deg
    per step; 1x1 mm patch at 5 um, stock z=0."""
    pitch = 0.005
    tool = ToolSpec("flat", 6.0, 2, [30.0], n_edge=50,
                    n_end=int(math.ceil(3.0 / (pitch / 2))))
    x0, y0, nx, ny = _patch(1.0, 1.0, pitch)
    px, py, spp = plan_passes(tool, 0.1, 0.5, nx * pitch, 0.0, 0.0, 1.0, pitch)
    proc = ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=0.5, ap=1.0, pass_x0=px, pass_y0=py,
                       steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx, ny=ny,
                       precision=precision)
    return Workload("slot_flat_d6", tool, proc)


def raster_ball_d10(precision: str = "fp32", width: float = 5.0, pitch: float = 0.001,
                    n_passes: int = 12, n_edge: int = 200, rot_step_deg: float = 0.1) -> Workload:
    """Ball end mill D=10, 4 flutes, helix 30 deg, radial runout 5 um at 30 deg,
    lead 15 / tilt 0; 12 parallel passes, fz=0.08, ae=0.3, 6000 rpm, ap=0.2
    (not stated by the configuration; chosen), 200 points along the edge,
    0.1 deg per step; 5x5 mm at 1 um. Keyword arguments shrink it for tests."""
    tool = ToolSpec("ball", 10.0, 4, [30.0], runout_mm=0.005, runout_phase_deg=30.0,
                    n_edge=n_edge)
    x0, y0, nx, ny = _patch(width, width, pitch)
    ae = 0.3
    first_y = -0.5 * (n_passes - 1) * ae
    px, py, spp = plan_passes(tool, 0.08, rot_step_deg, nx * pitch, 0.0, first_y, 0.2, pitch)
    proc = ProcessSpec(fz=0.08, rpm=6000, rot_step_deg=rot_step_deg, ap=0.2, pass_x0=px,
                       pass_y0=py, steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx,
                       ny=ny, n_passes=n_passes, ae=ae, lead_deg=15.0, precision=precision)
    return Workload("raster_ball_d10", tool, proc)


def plan_passes_dir(tool: ToolSpec, fz: float, rot_step_deg: float, width_x: float, width_y: float,
                    centre, n_passes: int, ae: float, ap: float, pitch: float, feed_dir_deg: float):
    """Tool path of a raster fed along feed_dir_deg: n_passes straight passes
    ae apart, centred on the patch across the feed and long enough along it
    that the whole tool clears the patch at both ends. Returns (pass_x0,
    pass_y0, steps_per_pass): the start of pass 0, about which the +X path is
    turned."""
    th = math.radians(feed_dir_deg)
    c, s = math.cos(th), math.sin(th)
    along = 0.5 * (width_x * abs(c) + width_y * abs(s))
    steps_per_rev = int(round(360.0 / rot_step_deg))
    feed_per_step = tool.n_teeth * fz / steps_per_rev
    overtravel = 0.5 * tool.diameter + tool.runout_mm + ap + 2.0 * pitch + tool.insert_radius
    half_steps = int(math.ceil((along + overtravel) / feed_per_step))
    a0 = -half_steps * feed_per_step
    b0 = -0.5 * (n_passes - 1) * ae
    return centre[0] + a0 * c - b0 * s, centre[1] + a0 * s + b0 * c, 2 * half_steps + 1


def raster_ball_tilted(precision: str = "fp32", width: float = 5.0, feed_dir_deg: float = 30.0,
                       pitch: float = 0.001, n_passes: Optional[int] = None, n_edge: int = 200,
                       rot_step_deg: float = 0.1, pass_mode: str = "one_way") -> Workload:
    """The ball raster's tool and cutting conditions fed at feed_dir_deg from
    +X (the lead leans the axis toward the feed): passes ae = 0.3 mm apart
    along the feed direction, enough of them to cross the square patch
    (n_passes overrides), on the same axis-aligned grid."""
    tool = ToolSpec("ball", 10.0, 4, [30.0], runout_mm=0.005, runout_phase_deg=30.0,
                    n_edge=n_edge)
    x0, y0, nx, ny = _patch(width, width, pitch)
    ae = 0.3
    th = math.radians(feed_dir_deg)
    if n_passes is None:
        across = nx * pitch * abs(math.sin(th)) + ny * pitch * abs(math.cos(th))
        n_passes = int(math.ceil(across / ae)) + 1
    px, py, spp = plan_passes_dir(tool, 0.08, rot_step_deg, nx * pitch, ny * pitch, (0.0, 0.0), n_passes, ae,
                                  0.2, pitch, feed_dir_deg)
    proc = ProcessSpec(fz=0.08, rpm=6000, rot_step_deg=rot_step_deg, ap=0.2, pass_x0=px,
                       pass_y0=py, steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx,
                       ny=ny, n_passes=n_passes, ae=ae, lead_deg=15.0, precision=precision,
                       pass_mode=pass_mode, feed_dir_deg=feed_dir_deg)
    return Workload("raster_ball_tilted", tool, proc)


def floor_flat_d12(seed: int = 2603, precision: str = "fp32", width: float = 20.0,
                   pitch: float = 0.002, rot_step_deg: float = 0.05) -> Workload:
    """Flat end mill D=12, 3 flutes with unequal helix 35/38/41 deg, runout
    8 um; floor finishing over 20x20 mm at 2 um, fz ~ U[0.04, 0.15] from the
    seed, 300 axial points, 0.05 deg per step. ap=0.5 and ae=0.4 D with passes
    covering the patch are chosen (not stated by the configuration)."""
    rng = np.random.default_rng(seed)
    fz = float(rng.uniform(0.04, 0.15))
    D = 12.0
    tool = ToolSpec("flat", D, 3, [35.0, 38.0, 41.0], runout_mm=0.008, runout_phase_deg=0.0,
                    n_edge=300, n_end=int(math.ceil((D / 2) / (pitch / 2))))
    x0, y0, nx, ny = _patch(width, width, pitch)
    ae = 0.4 * D
    n_passes = int(math.ceil((width + D) / ae))
    first_y = -0.5 * (n_passes - 1) * ae
    px, py, spp = plan_passes(tool, fz, rot_step_deg, nx * pitch, 0.0, first_y, 0.5, pitch)
    proc = ProcessSpec(fz=fz, rpm=6000, rot_step_deg=rot_step_deg, ap=0.5, pass_x0=px,
                       pass_y0=py, steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx,
                       ny=ny, n_passes=n_passes, ae=ae, precision=precision)
    return Workload("floor_flat_d12", tool, proc)


def side_wall_flat_d12(seed: int = 2603, precision: str = "fp32", length: float = 20.0, height: float = 1.0,
                       pitch: float = 0.002, rot_step_deg: float = 0.05, radial_depth: float = 0.3,
                       n_edge: Optional[int] = None) -> Workload:
    """The side of the side-plus-floor finish: the wall the flank of the
    floor_flat_d12 tool (flat D=12, 3 flutes 35/38/41 deg, runout 8 um, the
    same seeded fz) leaves on the +Y side of one pass along +X, taking a
    radial depth of 0.3 mm and ap = `height`. Map: length x height at 2 um
    over x and z, height -y. Flank points every pitch/2 along the axis (so
    every row of the map holds a sample), 0.05 deg per step."""
    rng = np.random.default_rng(seed)
    fz = float(rng.uniform(0.04, 0.15))
    D = 12.0
    if n_edge is None:
        n_edge = int(math.ceil(height / (pitch / 2))) + 1
    tool = ToolSpec("flat", D, 3, [35.0, 38.0, 41.0], runout_mm=0.008, runout_phase_deg=0.0, n_edge=n_edge,
                    n_end=0)
    nx = int(round(length / pitch))
    ny = int(round(height / pitch))
    x0 = -0.5 * nx * pitch + CELL_OFFSET[0] * pitch
    y0 = -height + CELL_OFFSET[1] * pitch   # map rows run over z from the tool tip up
    px, py, spp = plan_passes(tool, fz, rot_step_deg, nx * pitch, 0.0, 0.0, height, pitch)
    proc = ProcessSpec(fz=fz, rpm=6000, rot_step_deg=rot_step_deg, ap=height, pass_x0=px, pass_y0=py,
                       steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx, ny=ny, precision=precision,
                       surface="wall", wall_y=0.5 * D - radial_depth)
    return Workload("side_wall_flat_d12", tool, proc)


# Case 2 of the paper (Section 4.2.1): face mill R217.29-2520.3-05.2.070,
# cutting diameter 10 mm, two round inserts of radius 5 mm, radial rake 0.6,
# axial rake 0; (vc m/min, fz mm, ap mm, eps_r mm, eps_a mm) per case
PAPER_CASES = [(170, 0.6, 0.5, 0.011, 0.003), (200, 0.4, 0.4, -0.026, 0.009), (230, 0.5, 0.3, -0.013, 0.007)]
# the nine conditions of the computational-performance study (Section 4.3),
# 10 x 5 mm, zero run-out: (vc, fz, ap)
PAPER_GRID = [(170, 0.4, 0.3), (170, 0.5, 0.4), (170, 0.6, 0.5), (200, 0.4, 0.3), (200, 0.5, 0.4),
              (200, 0.6, 0.5), (230, 0.4, 0.3), (230, 0.5, 0.4), (230, 0.6, 0.5)]


def paper_insert_tool(eps_r: float = 0.0, eps_a: float = 0.0, n_edge: int = 100) -> ToolSpec:
    return ToolSpec("insert", 10.0, 2, [0.0], n_edge=n_edge, insert_radius=5.0, rake_f_deg=0.6, rake_p_deg=0.0,
                    eps_r_mm=eps_r, eps_a_mm=eps_a)


def face_mill_insert(vc: float, fz: float, ap: float, eps_r: float = 0.0, eps_a: float = 0.0,
                     precision: str = "fp32", pitch: float = 0.005, length: float = 10.0, width: float = 5.0,
                     rot_step_deg: float = 0.1, n_edge: int = 100, dt_s: Optional[float] = None) -> Workload:
    """One face-milling pass of the paper's insert cutter over a length x
    width patch (feed along +X through the patch centre). The grid pitch,
    angle step and edge-point count are not stated by the paper (chosen);
    rpm follows from vc and the 10 mm cutting diameter.

    dt_s=None: fixed angle step rot_step_deg, and the pass overruns the patch
    so the whole cutter clears it (rpm then labels time only).
    dt_s given: fixed time step, as the paper's performance study implies --
    its trajectory-point counts equal (tool-centre travel) / (vf * dt) with a
    travel of the patch length (Section 4.3 table; 2e-7 s reproduces them).
    The angle step is the nearest one with a whole number of steps per
    revolution, and the tool centre runs from the patch's start to its end."""
    tool = paper_insert_tool(eps_r, eps_a, n_edge)
    rpm = 1000.0 * vc / (math.pi * tool.diameter)
    x0, y0, nx, ny = _patch(length, width, pitch)
    if dt_s is None:
        px, py, spp = plan_passes(tool, fz, rot_step_deg, nx * pitch, 0.0, 0.0, ap, pitch)
    else:
        steps_per_rev = int(round(60.0 / (rpm * dt_s)))
        rot_step_deg = 360.0 / steps_per_rev
        feed_per_step = tool.n_teeth * fz / steps_per_rev
        spp = int(round(nx * pitch / feed_per_step))
        px, py = x0 - CELL_OFFSET[0] * pitch, 0.0
    proc = ProcessSpec(fz=fz, rpm=rpm, rot_step_deg=rot_step_deg, ap=ap, pass_x0=px, pass_y0=py,
                       steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch, nx=nx, ny=ny, precision=precision)
    return Workload("face_mill_vc%g_fz%g_ap%g" % (vc, fz, ap), tool, proc)


def paper_case(i: int, **kw) -> Workload:
    vc, fz, ap, er, ea = PAPER_CASES[i]
    return face_mill_insert(vc, fz, ap, er, ea, **kw)


def paper_grid(**kw) -> List[Workload]:
    return [face_mill_insert(vc, fz, ap, **kw) for vc, fz, ap in PAPER_GRID]


def _lhs(rng: np.random.Generator, n: int, dims: int) -> np.ndarray:
    """Latin hypercube sample in [0,1)^dims: one point per stratum per axis."""
    u = rng.random((n, dims))
    out = np.empty((n, dims))
    for d in range(dims):
        out[:, d] = (rng.permutation(n) + u[:, d]) / n
    return out


def lhs_batch(n: int = 4096, seed: int = 4096, precision: str = "fp32",
              rot_step_deg: float = 0.1, n_edge: int = 200,
              side_range=(0.5, 4.0), pitch_range_um=(1.0, 5.0)) -> List[Workload]:
    """Seeded Latin-hypercube batch: ball or flat end, D in [4,16] mm, 2-6
    flutes, helix [20,45] deg, runout [0,15] um with phase [0,360), lead and
    tilt [0,20] deg, fz [0.03,0.2] mm, ae [0.1,1.0] mm; square patches 0.5-4 mm
    at 1-5 um pitch; 0.1 deg per step and 200 edge points (chosen). Depth of
    cut ap = 0.2 mm (chosen); passes cover the patch."""
    rng = np.random.default_rng(seed)
    X = _lhs(rng, n, 12)
    out = []
    for i in range(n):
        x = X[i]
        kind = "ball" if x[0] < 0.5 else "flat"
        D = 4.0 + 12.0 * x[1]
        N = 2 + int(x[2] * 5)
        helix = 20.0 + 25.0 * x[3]
        runout = 0.015 * x[4]
        rphase = 360.0 * x[5]
        lead = 20.0 * x[6]
        tilt = 20.0 * x[7]
        fz = 0.03 + 0.17 * x[8]
        ae = 0.1 + 0.9 * x[9]
        side = side_range[0] + (side_range[1] - side_range[0]) * x[10]
        pitch = 1e-3 * (pitch_range_um[0] + (pitch_range_um[1] - pitch_range_um[0]) * x[11])
        ap = 0.2
        n_end = int(math.ceil((D / 2) / (pitch / 2))) if kind == "flat" else 0
        tool = ToolSpec(kind, D, N, [helix], runout_mm=runout, runout_phase_deg=rphase,
                        n_edge=n_edge, n_end=n_end)
        x0, y0, nx, ny = _patch(side, side, pitch)
        n_passes = int(math.ceil(side / ae)) + 1
        # a tilted flat end cuts with the low side of its rim, D/2 from the
        # axis toward (+lead, +tilt): shift the tool path so that rim sweeps
        # the patch
        sx = sy = 0.0
        if kind == "flat" and (lead > 0.0 or tilt > 0.0):
            a, b = math.sin(math.radians(lead)), math.sin(math.radians(tilt))
            nrm = math.hypot(a, b)
            sx, sy = 0.5 * D * a / nrm, 0.5 * D * b / nrm
        first_y = -0.5 * (n_passes - 1) * ae - sy
        px, py, spp = plan_passes(tool, fz, rot_step_deg, nx * pitch, -sx, first_y, ap, pitch)
        proc = ProcessSpec(fz=fz, rpm=6000, rot_step_deg=rot_step_deg, ap=ap, pass_x0=px,
                           pass_y0=py, steps_per_pass=spp, x0=x0, y0=y0, pitch=pitch,
                           nx=nx, ny=ny, n_passes=n_passes, ae=ae, lead_deg=lead,
                           tilt_deg=tilt, precision=precision)
        out.append(Workload("lhs_%d" % i, tool, proc))
    return out


def serve_stream(n: int, seed: int = 5, fp64_fraction: float = 0.3, rot_step_deg: float = 0.1,
                 n_edge: int = 200, cells_range=(0.25e6, 25e6), n_setups: Optional[int] = None) -> List[Workload]:
    """Requests of a served stream: tools and cutting conditions drawn from
    the batch distribution (seeded Latin hypercube), square patches whose
    cell count is log-uniform in [0.25, 25] Mcells at 1-5 um pitch, and a
    seeded 30 % of the requests in FP64 (the rest FP32).

    n_setups: None draws every request's tool and set-up afresh. A number
    draws them from a seeded catalogue of that many set-ups -- tool, depth of
    cut, lead, tilt, step angle and pitch, as a dataset generator sweeping
    feeds and step-overs over a fixed tool set would -- while feed,
    step-over, patch size and precision stay per request."""
    rng = np.random.default_rng(seed + 1000)
    base = lhs_batch(n=n, seed=seed, rot_step_deg=rot_step_deg, n_edge=n_edge)
    if n_setups is not None:
        cat = lhs_batch(n=n_setups, seed=seed + 7, rot_step_deg=rot_step_deg, n_edge=n_edge)
        pick = np.random.default_rng(seed + 2000).integers(0, n_setups, size=n)
        mixed = []
        for w, k in zip(base, pick):
            c = cat[int(k)]
            mixed.append(Workload(w.name, c.tool, w.process.replace(
                ap=c.process.ap, lead_deg=c.process.lead_deg, tilt_deg=c.process.tilt_deg,
                rot_step_deg=c.process.rot_step_deg, pitch=c.process.pitch, phase0_deg=c.process.phase0_deg)))
        base = mixed
    out = []
    for w in base:
        t, p = w.tool, w.process
        cells = float(np.exp(rng.uniform(np.log(cells_range[0]), np.log(cells_range[1]))))
        side_cells = int(round(np.sqrt(cells)))
        side = side_cells * p.pitch
        if t.kind == "flat":
            t = dataclasses.replace(t, n_end=int(math.ceil((t.diameter / 2) / (p.pitch / 2))))
        x0, y0, nx, ny = _patch(side, side, p.pitch)
        n_passes = int(math.ceil(side / p.ae)) + 1
        sx = sy = 0.0
        if t.kind == "flat" and (p.lead_deg > 0.0 or p.tilt_deg > 0.0):
            a, b = math.sin(math.radians(p.lead_deg)), math.sin(math.radians(p.tilt_deg))
            nrm = math.hypot(a, b)
            sx, sy = 0.5 * t.diameter * a / nrm, 0.5 * t.diameter * b / nrm
        first_y = -0.5 * (n_passes - 1) * p.ae - sy
        px, py, spp = plan_passes(t, p.fz, p.rot_step_deg, nx * p.pitch, -sx, first_y, p.ap, p.pitch)
        prec = "fp64" if rng.random() < fp64_fraction else "fp32"
        p2 = p.replace(x0=x0, y0=y0, nx=nx, ny=ny, n_passes=n_passes, pass_x0=px, pass_y0=py,
                       steps_per_pass=spp, precision=prec)
        out.append(Workload("serve_%d" % len(out), t, p2))
    return out


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 5) -> np.ndarray:
    """Seeded Poisson process: arrival times (s) of n requests."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def mixed_precision(workloads: List[Workload], fp64_fraction: float = 0.3,
                    seed: int = 6) -> List[Workload]:
    """Mark a seeded fraction of the requests as FP64, the rest FP32."""
    rng = np.random.default_rng(seed)
    out = []
    for w in workloads:
        prec = "fp64" if rng.random() < fp64_fraction else "fp32"
        out.append(Workload(w.name, w.tool, w.process.replace(precision=prec), w.note))
    return out
