"""ctypes front end of the plain FP64 CPU oracle (test infrastructure).

Only tests/, the smoke check and the CPU-baseline leg of bench.py import this
module. It converts the seeded workload parameters into the oracle's own C
structs and returns NumPy arrays. No code here is shared with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build_oracle

MAX_TEETH = 16
MAX_PROFILES = 16


class OrcTool(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n_teeth", C.c_int32), ("n_edge", C.c_int32), ("n_end", C.c_int32),
        ("diameter", C.c_double),
        ("helix_deg", C.c_double * MAX_TEETH), ("tooth_deg", C.c_double * MAX_TEETH),
        ("runout_mm", C.c_double), ("runout_phase_deg", C.c_double),
        ("insert_radius", C.c_double), ("rake_f_deg", C.c_double), ("rake_p_deg", C.c_double),
        ("eps_r_mm", C.c_double), ("eps_a_mm", C.c_double), ("corner_radius", C.c_double),
    ]


class OrcProcess(C.Structure):
    _fields_ = [
        ("fz", C.c_double), ("rot_step_deg", C.c_double), ("phase0_deg", C.c_double),
        ("rot_sense", C.c_int32), ("n_passes", C.c_int32),
        ("ap", C.c_double), ("lead_deg", C.c_double), ("tilt_deg", C.c_double),
        ("ae", C.c_double), ("pass_x0", C.c_double), ("pass_y0", C.c_double),
        ("steps_per_pass", C.c_int64), ("stock_z", C.c_double),
        ("x0", C.c_double), ("y0", C.c_double), ("pitch", C.c_double),
        ("nx", C.c_int32), ("ny", C.c_int32), ("z_ref_override", C.c_double),
        ("surface", C.c_int32), ("wall_y", C.c_double), ("pass_mode", C.c_int32),
        ("feed_dir_deg", C.c_double),
    ]


class OrcStats(C.Structure):
    _fields_ = [
        ("trajectory_points", C.c_int64), ("landed", C.c_int64), ("cutting", C.c_int64),
        ("cells_hit", C.c_int64), ("cells_flagged", C.c_int64), ("z_ref", C.c_double),
    ]


class OrcRough(C.Structure):
    _fields_ = [
        ("n", C.c_double), ("mean", C.c_double), ("zmin", C.c_double), ("zmax", C.c_double),
        ("Sa", C.c_double), ("Sq", C.c_double), ("Sp", C.c_double), ("Sv", C.c_double),
        ("Sz", C.c_double), ("Ssk", C.c_double), ("Sku", C.c_double),
        ("n_rows", C.c_int32), ("n_cols", C.c_int32),
        ("row_index", C.c_int32 * MAX_PROFILES), ("col_index", C.c_int32 * MAX_PROFILES),
        ("Ra_row", C.c_double * MAX_PROFILES), ("Rz_row", C.c_double * MAX_PROFILES),
        ("Ra_col", C.c_double * MAX_PROFILES), ("Rz_col", C.c_double * MAX_PROFILES),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.orc_points_per_tooth.argtypes = [P(OrcTool), C.c_int]
        L.orc_edge_points.argtypes = [P(OrcTool), P(OrcProcess), C.c_int, P(C.c_double), C.c_int]
        L.orc_z_ref.argtypes = [P(OrcTool), P(OrcProcess), C.c_int]
        L.orc_z_ref.restype = C.c_double
        L.orc_pose.argtypes = [P(OrcTool), P(OrcProcess), C.c_int64, C.c_int, C.c_int, P(C.c_double)]
        L.orc_fsm.argtypes = [P(OrcTool), P(OrcProcess), P(C.c_double), P(C.c_uint8), P(OrcStats),
                              C.c_int]
        L.orc_gather.argtypes = [P(OrcTool), P(OrcProcess), C.c_int, C.c_int, C.c_int, C.c_int,
                                 C.c_int, P(C.c_double)]
        L.orc_trajectory.argtypes = [P(OrcTool), P(OrcProcess), C.c_int64, C.c_int64, P(C.c_double),
                                     P(C.c_int32)]
        L.orc_gauss_filter.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double, P(C.c_double)]
        L.orc_sl_surface.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                     P(C.c_double)]
        L.orc_roughness.argtypes = [P(C.c_double), C.c_int, C.c_int, C.c_int, C.c_int, P(OrcRough)]
        _lib = L
    return _lib


def make_tool(tool) -> OrcTool:
    t = OrcTool()
    t.kind = {"flat": 0, "ball": 1, "insert": 2, "torus": 3}[tool.kind]
    t.n_teeth = tool.n_teeth
    t.n_edge = tool.n_edge
    t.n_end = tool.n_end if tool.kind in ("flat", "torus") else 0
    t.diameter = tool.diameter
    for k, (h, a) in enumerate(zip(tool.helix(), tool.teeth_angles())):
        t.helix_deg[k] = h
        t.tooth_deg[k] = a
    t.runout_mm = tool.runout_mm
    t.runout_phase_deg = tool.runout_phase_deg
    t.insert_radius = tool.insert_radius
    t.rake_f_deg = tool.rake_f_deg
    t.rake_p_deg = tool.rake_p_deg
    t.eps_r_mm = tool.eps_r_mm
    t.eps_a_mm = tool.eps_a_mm
    t.corner_radius = tool.corner_radius
    return t


def make_process(proc, z_ref=None) -> OrcProcess:
    p = OrcProcess()
    for name in ("fz", "rot_step_deg", "phase0_deg", "rot_sense", "n_passes", "ap", "lead_deg",
                 "tilt_deg", "ae", "pass_x0", "pass_y0", "steps_per_pass", "stock_z", "x0", "y0",
                 "pitch", "nx", "ny"):
        setattr(p, name, getattr(proc, name))
    p.z_ref_override = math.nan if z_ref is None else z_ref
    p.surface = {"floor": 0, "wall": 1}[proc.surface]
    p.wall_y = proc.wall_y
    p.pass_mode = {"one_way": 0, "zigzag": 1}[proc.pass_mode]
    p.feed_dir_deg = proc.feed_dir_deg
    return p


@dataclass
class FsmResult:
    H: np.ndarray          # [ny, nx] float64
    flags: np.ndarray      # [ny, nx] bool: next to a boundary-tie point
    stats: dict


def fsm(workload, n_threads: int = 1, z_ref=None) -> FsmResult:
    """Plain scatter FSM of the whole tool path."""
    t, p = make_tool(workload.tool), make_process(workload.process, z_ref)
    H = np.empty((p.ny, p.nx), np.float64)
    F = np.zeros((p.ny, p.nx), np.uint8)
    st = OrcStats()
    rc = lib().orc_fsm(C.byref(t), C.byref(p), H.ctypes.data_as(C.POINTER(C.c_double)),
                       F.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(st), int(n_threads))
    if rc != 0:
        raise ValueError("oracle rejected the workload")
    stats = {k: getattr(st, k) for k, _ in OrcStats._fields_}
    return FsmResult(H, F.astype(bool), stats)


def gather(workload, refine: int = 1, window=None, z_ref=None) -> np.ndarray:
    """Brute-force per-cell inverse over the refine-times denser sample set.
    window = (i0, k0, ni, nk); default the whole grid."""
    t, p = make_tool(workload.tool), make_process(workload.process, z_ref)
    if window is None:
        window = (0, 0, p.nx, p.ny)
    i0, k0, ni, nk = window
    Hw = np.empty((nk, ni), np.float64)
    rc = lib().orc_gather(C.byref(t), C.byref(p), int(refine), i0, k0, ni, nk,
                          Hw.ctypes.data_as(C.POINTER(C.c_double)))
    if rc != 0:
        raise ValueError("oracle rejected the workload")
    return Hw


def edge_points(workload, refine: int = 1) -> np.ndarray:
    """Tool-frame edge points, shape [n_teeth, points_per_tooth, 3]."""
    t, p = make_tool(workload.tool), make_process(workload.process)
    E = lib().orc_points_per_tooth(C.byref(t), refine)
    out = np.empty((t.n_teeth, E, 3), np.float64)
    n = lib().orc_edge_points(C.byref(t), C.byref(p), refine,
                              out.ctypes.data_as(C.POINTER(C.c_double)), out.size // 3)
    if n < 0:
        raise ValueError("oracle rejected the workload")
    return out


def z_ref(workload, refine: int = 1) -> float:
    t, p = make_tool(workload.tool), make_process(workload.process)
    return lib().orc_z_ref(C.byref(t), C.byref(p), refine)


def pose(workload, s: int, K: int, j: int) -> np.ndarray:
    t, p = make_tool(workload.tool), make_process(workload.process)
    w = (C.c_double * 3)()
    if lib().orc_pose(C.byref(t), C.byref(p), int(s), int(K), int(j), w) != 0:
        raise ValueError("bad pose request")
    return np.array(list(w))


def trajectory(workload, s0: int = 0, count=None, z_ref=None):
    """Lowest point of every cutting edge at global steps s0 .. s0+count-1:
    returns (xyz [count, n_teeth, 3] float64, j [count, n_teeth] int32)."""
    t, p = make_tool(workload.tool), make_process(workload.process, z_ref)
    total = p.n_passes * p.steps_per_pass
    if count is None:
        count = total - s0
    xyz = np.empty((count, t.n_teeth, 3), np.float64)
    j = np.empty((count, t.n_teeth), np.int32)
    rc = lib().orc_trajectory(C.byref(t), C.byref(p), int(s0), int(count),
                              xyz.ctypes.data_as(C.POINTER(C.c_double)), j.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise ValueError("oracle rejected the request")
    return xyz, j


def gauss_filter(H: np.ndarray, pitch: float, lam: float) -> np.ndarray:
    """ISO 16610-61 Gaussian low-pass of H (cutoff lam), zero-order end correction."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    ny, nx = H.shape
    out = np.empty_like(H)
    if lib().orc_gauss_filter(H.ctypes.data_as(C.POINTER(C.c_double)), nx, ny, float(pitch), float(lam),
                              out.ctypes.data_as(C.POINTER(C.c_double))) != 0:
        raise ValueError("bad filter request")
    return out


def sl_surface(H: np.ndarray, pitch: float, lambda_s: float, lambda_c: float) -> np.ndarray:
    """S-filter (lambda_s) then remove the L-filter mean surface (lambda_c)."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    ny, nx = H.shape
    out = np.empty_like(H)
    if lib().orc_sl_surface(H.ctypes.data_as(C.POINTER(C.c_double)), nx, ny, float(pitch), float(lambda_s),
                            float(lambda_c), out.ctypes.data_as(C.POINTER(C.c_double))) != 0:
        raise ValueError("bad filter request")
    return out


def roughness(H: np.ndarray, n_rows: int = 10, n_cols: int = 10) -> dict:
    H = np.ascontiguousarray(H, dtype=np.float64)
    ny, nx = H.shape
    r = OrcRough()
    rc = lib().orc_roughness(H.ctypes.data_as(C.POINTER(C.c_double)), nx, ny, n_rows, n_cols,
                             C.byref(r))
    if rc != 0:
        raise ValueError("bad roughness request")
    out = {k: getattr(r, k) for k in ("n", "mean", "zmin", "zmax", "Sa", "Sq", "Sp", "Sv", "Sz",
                                      "Ssk", "Sku")}
    out["row_index"] = list(r.row_index)[:n_rows]
    out["col_index"] = list(r.col_index)[:n_cols]
    out["Ra_row"] = np.array(r.Ra_row[:n_rows])
    out["Rz_row"] = np.array(r.Rz_row[:n_rows])
    out["Ra_col"] = np.array(r.Ra_col[:n_cols])
    out["Rz_col"] = np.array(r.Rz_col[:n_cols])
    return out
