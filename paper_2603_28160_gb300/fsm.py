"""Thin Python binding of the C ABI in include/fsm.h (argument marshalling only).

Every step of the surface generation runs in the CUDA kernels of libfsm.so;
this module converts ToolSpec / ProcessSpec into the C descriptors, passes
torch tensors' device pointers and streams, and unpacks results. There is no
CPU fallback: if libfsm.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

from .workloads import ProcessSpec, ToolSpec, Workload

MAX_TEETH = 16
MAX_PROFILES = 16
FSM_OK, FSM_PENDING = 0, 1
FSM_FP64, FSM_FP32 = 0, 1
_STATUS = {0: "FSM_OK", 1: "FSM_PENDING", -1: "FSM_E_INVALID", -2: "FSM_E_NOMEM", -3: "FSM_E_CUDA",
           -4: "FSM_E_TIMEOUT", -5: "FSM_E_CANCELLED", -6: "FSM_E_STATE"}

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsm.so")


class ToolDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_teeth", C.c_int32), ("n_edge", C.c_int32), ("n_end", C.c_int32),
                ("diameter", C.c_double), ("helix_deg", C.c_double * MAX_TEETH),
                ("tooth_deg", C.c_double * MAX_TEETH), ("runout_mm", C.c_double),
                ("runout_phase_deg", C.c_double), ("insert_radius", C.c_double), ("rake_f_deg", C.c_double),
                ("rake_p_deg", C.c_double), ("eps_r_mm", C.c_double), ("eps_a_mm", C.c_double),
                ("corner_radius", C.c_double)]


class ProcessDesc(C.Structure):
    _fields_ = [("fz", C.c_double), ("rpm", C.c_double), ("rot_step_deg", C.c_double),
                ("phase0_deg", C.c_double), ("rot_sense", C.c_int32), ("n_passes", C.c_int32),
                ("ap", C.c_double), ("lead_deg", C.c_double), ("tilt_deg", C.c_double), ("ae", C.c_double),
                ("pass_x0", C.c_double), ("pass_y0", C.c_double), ("steps_per_pass", C.c_int64),
                ("stock_z", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("pitch", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32), ("precision", C.c_int32), ("surface", C.c_int32),
                ("wall_y", C.c_double), ("pass_mode", C.c_int32), ("reserved", C.c_int32),
                ("feed_dir_deg", C.c_double)]


class PredictOpts(C.Structure):
    _fields_ = [("tile_x", C.c_int32), ("tile_y", C.c_int32), ("block_threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("d_counters", C.c_void_p), ("sweep_events", C.c_void_p * 2),
                ("sweep_form", C.c_int32), ("reserved", C.c_int32), ("d_form_tasks", C.c_void_p)]


FORMS = {"auto": 0, "item": 1, "phase": 2}


class RoughnessOut(C.Structure):
    _fields_ = [("n", C.c_double), ("mean", C.c_double), ("zmin", C.c_double), ("zmax", C.c_double),
                ("Sa", C.c_double), ("Sq", C.c_double), ("Sp", C.c_double), ("Sv", C.c_double),
                ("Sz", C.c_double), ("Ssk", C.c_double), ("Sku", C.c_double),
                ("n_rows", C.c_int32), ("n_cols", C.c_int32),
                ("row_index", C.c_int32 * MAX_PROFILES), ("col_index", C.c_int32 * MAX_PROFILES),
                ("Ra_row", C.c_double * MAX_PROFILES), ("Rz_row", C.c_double * MAX_PROFILES),
                ("Ra_col", C.c_double * MAX_PROFILES), ("Rz_col", C.c_double * MAX_PROFILES)]


class Result(C.Structure):
    _fields_ = [("d_heights", C.c_void_p), ("precision", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
                ("status", C.c_int32), ("rough", RoughnessOut), ("queue_s", C.c_double),
                ("latency_s", C.c_double)]


class ServerInfo(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("cancelled", C.c_uint64),
                ("failed", C.c_uint64), ("batches", C.c_uint64), ("table_hits", C.c_uint64),
                ("table_misses", C.c_uint64), ("bytes_in_use", C.c_uint64), ("bytes_peak", C.c_uint64),
                ("table_bytes", C.c_uint64), ("queue_depth", C.c_int32), ("queue_peak", C.c_int32),
                ("tables_cached", C.c_int32), ("reserved", C.c_int32)]


class BatchInterval(C.Structure):
    _fields_ = [("slot", C.c_int32), ("n_requests", C.c_int32), ("t_start_ms", C.c_double),
                ("t_end_ms", C.c_double)]


ROUGH_BYTES = C.sizeof(RoughnessOut)

# (name, argtypes) of every exported function; all return fsm_status (int)
_P = C.c_void_p
SIGNATURES = {
    "fsm_create_context": [C.c_int, C.POINTER(_P)],
    "fsm_destroy_context": [_P],
    "fsm_create_tool": [_P, C.POINTER(ToolDesc), C.POINTER(_P)],
    "fsm_destroy_tool": [_P, _P],
    "fsm_set_process": [_P, C.POINTER(ProcessDesc), C.POINTER(_P)],
    "fsm_destroy_process": [_P, _P],
    "fsm_predict_surface": [_P, _P, _P, _P, C.POINTER(PredictOpts), _P],
    "fsm_roughness": [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P],
    "fsm_roughness_noalloc": [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P],
    "fsm_predict_batch": [_P, C.c_int32, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), _P,
                          C.POINTER(PredictOpts), _P],
    "fsm_autotune": [_P, _P, _P, _P, C.c_int32, C.POINTER(PredictOpts), C.POINTER(C.c_float), _P],
    "fsm_batch_create": [_P, C.c_int32, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P), _P,
                         C.POINTER(PredictOpts), C.POINTER(_P)],
    "fsm_batch_run": [_P, _P, _P],
    "fsm_batch_destroy": [_P, _P],
    "fsm_server_start": [_P, C.c_size_t, C.c_int32, C.c_int32],
    "fsm_server_stop": [_P],
    "fsm_submit": [_P, _P, _P, C.POINTER(C.c_uint64)],
    "fsm_poll": [_P, C.c_uint64, C.c_int32, C.POINTER(Result)],
    "fsm_release_result": [_P, C.c_uint64],
    "fsm_cancel": [_P, C.c_uint64],
    "fsm_server_stats": [_P, C.POINTER(ServerInfo)],
    "fsm_server_batches": [_P, C.POINTER(BatchInterval), C.c_int32, C.POINTER(C.c_int32)],
    "fsm_server_inject_alloc_failures": [_P, C.c_int32],
    "fsm_predict_trajectory": [_P, _P, _P, _P, C.c_int64, _P],
    "fsm_trajectory_records": [_P, _P, C.POINTER(C.c_int64)],
    "fsm_filter": [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, _P, _P],
    "fsm_moment_partials": [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_double, _P, _P],
}

_lib = None


class FsmError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__("%s -> %s: %s" % (fn, _STATUS.get(status, status), msg))
        self.status = status


def lib() -> C.CDLL:
    """Load libfsm.so; raise if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfsm.so is not built; run paper_2603_28160_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.fsm_last_error.argtypes = [_P]
        L.fsm_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def tool_desc(t: ToolSpec) -> ToolDesc:
    d = ToolDesc()
    d.kind = {"flat": 0, "ball": 1, "insert": 2, "torus": 3}[t.kind]
    d.n_teeth = t.n_teeth
    d.n_edge = t.n_edge
    d.n_end = t.n_end if t.kind in ("flat", "torus") else 0
    d.diameter = t.diameter
    for k, (h, a) in enumerate(zip(t.helix(), t.teeth_angles())):
        d.helix_deg[k] = h
        d.tooth_deg[k] = a
    d.runout_mm = t.runout_mm
    d.runout_phase_deg = t.runout_phase_deg
    d.insert_radius = t.insert_radius
    d.rake_f_deg = t.rake_f_deg
    d.rake_p_deg = t.rake_p_deg
    d.eps_r_mm = t.eps_r_mm
    d.eps_a_mm = t.eps_a_mm
    d.corner_radius = t.corner_radius
    return d


def process_desc(p: ProcessSpec) -> ProcessDesc:
    d = ProcessDesc()
    for name in ("fz", "rpm", "rot_step_deg", "phase0_deg", "rot_sense", "n_passes", "ap", "lead_deg",
                 "tilt_deg", "ae", "pass_x0", "pass_y0", "steps_per_pass", "stock_z", "x0", "y0", "pitch",
                 "nx", "ny"):
        setattr(d, name, getattr(p, name))
    d.precision = {"fp64": FSM_FP64, "fp32": FSM_FP32}[p.precision]
    d.surface = {"floor": 0, "wall": 1}[p.surface]
    d.wall_y = p.wall_y
    d.pass_mode = {"one_way": 0, "zigzag": 1}[p.pass_mode]
    d.feed_dir_deg = p.feed_dir_deg
    return d


def rough_dict(r: RoughnessOut) -> dict:
    out = {k: getattr(r, k) for k in ("n", "mean", "zmin", "zmax", "Sa", "Sq", "Sp", "Sv", "Sz", "Ssk", "Sku")}
    nr, nc = r.n_rows, r.n_cols
    out["row_index"] = list(r.row_index)[:nr]
    out["col_index"] = list(r.col_index)[:nc]
    out["Ra_row"] = np.array(r.Ra_row[:nr])
    out["Rz_row"] = np.array(r.Rz_row[:nr])
    out["Ra_col"] = np.array(r.Ra_col[:nc])
    out["Rz_col"] = np.array(r.Rz_col[:nc])
    return out


def _stream_ptr(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class _Handle:
    def __init__(self, ctx: "Context", ptr: int, destroy: str):
        self.ctx, self.ptr, self._destroy = ctx, ptr, destroy

    def close(self):
        if self.ptr:
            getattr(lib(), self._destroy)(self.ctx.ptr, self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A library context on one CUDA device (fsm_create_context)."""

    def __init__(self, device: int = 0):
        self.ptr = None
        p = _P()
        self._call("fsm_create_context", int(device), C.byref(p))
        self.ptr = p.value
        self.device = device

    def _call(self, fn: str, *args) -> int:
        rc = getattr(lib(), fn)(*args)
        if rc not in (FSM_OK, FSM_PENDING):
            msg = lib().fsm_last_error(self.ptr).decode(errors="replace")
            raise FsmError(fn, rc, msg)
        return rc

    def close(self):
        if self.ptr:
            lib().fsm_destroy_context(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- handles ----------------------------------------------------------
    def tool(self, spec: ToolSpec) -> _Handle:
        d = tool_desc(spec)
        p = _P()
        self._call("fsm_create_tool", self.ptr, C.byref(d), C.byref(p))
        return _Handle(self, p.value, "fsm_destroy_tool")

    def process(self, spec: ProcessSpec) -> _Handle:
        d = process_desc(spec)
        p = _P()
        self._call("fsm_set_process", self.ptr, C.byref(d), C.byref(p))
        return _Handle(self, p.value, "fsm_destroy_process")

    # -- single surface ---------------------------------------------------
    @staticmethod
    def _opts(tile=None, threads=None, counters=None, events=None, ctas_per_sm=None, form=None,
              form_tasks=None) -> Optional[PredictOpts]:
        if (tile is None and threads is None and counters is None and events is None and ctas_per_sm is None
                and form is None and form_tasks is None):
            return None
        o = PredictOpts()
        if form is not None:
            o.sweep_form = FORMS[form]
        if form_tasks is not None:  # CUDA int64 tensor of 2: tasks in the item and the phase form
            o.d_form_tasks = form_tasks.data_ptr()
        if tile is not None:
            o.tile_x, o.tile_y = int(tile[0]), int(tile[1])
        if threads is not None:
            o.block_threads = int(threads)
        if ctas_per_sm is not None:
            o.ctas_per_sm = int(ctas_per_sm)
        if counters is not None:
            o.d_counters = counters.data_ptr()
        if events is not None:  # two torch.cuda.Event objects, already recorded once
            o.sweep_events[0] = events[0].cuda_event
            o.sweep_events[1] = events[1].cuda_event
        return o

    def predict_surface(self, tool: _Handle, proc: _Handle, out, tile=None, threads=None, counters=None,
                        stream=None, events=None, ctas_per_sm=None, form=None, form_tasks=None) -> None:
        """Enqueue fsm_predict_surface writing into the CUDA tensor `out`.
        events: optional pair of torch.cuda.Event recorded around the sweep;
        form: "auto", "item" or "phase" (fsm_predict_opts.sweep_form)."""
        o = self._opts(tile, threads, counters, events, ctas_per_sm, form, form_tasks)
        self._call("fsm_predict_surface", self.ptr, tool.ptr, proc.ptr, out.data_ptr(),
                   C.byref(o) if o is not None else None, _stream_ptr(stream))

    def trajectory(self, tool: _Handle, proc: _Handle, out=None, stream=None):
        """fsm_predict_trajectory into a CUDA uint8 tensor of [records, 32]
        bytes (allocated if out is None); see trajectory_views()."""
        n = C.c_int64()
        self._call("fsm_trajectory_records", tool.ptr, proc.ptr, C.byref(n))
        if out is None:
            import torch
            out = torch.empty((n.value, TRAJ_BYTES), dtype=torch.uint8, device="cuda")
        self._call("fsm_predict_trajectory", self.ptr, tool.ptr, proc.ptr, out.data_ptr(),
                   out.numel() // TRAJ_BYTES, _stream_ptr(stream))
        return out

    def filter(self, heights, pitch: float, lambda_s: float, lambda_c: float, out=None, stream=None):
        """fsm_filter: ISO Gaussian S-filter (lambda_s) and L-filter
        (lambda_c) of a CUDA height map; returns the SL-surface tensor."""
        import torch
        ny, nx = heights.shape
        prec = FSM_FP64 if heights.dtype == torch.float64 else FSM_FP32
        if out is None:
            out = torch.empty_like(heights)
        self._call("fsm_filter", self.ptr, heights.data_ptr(), prec, nx, ny, float(pitch), float(lambda_s),
                   float(lambda_c), out.data_ptr(), _stream_ptr(stream))
        return out

    def autotune(self, tool: _Handle, proc: _Handle, out, max_candidates: int = 0, stream=None) -> dict:
        """fsm_autotune: time sweep configurations on this workload; the
        choice is also recorded in the context for later predictions."""
        best = PredictOpts()
        ms = C.c_float()
        self._call("fsm_autotune", self.ptr, tool.ptr, proc.ptr, out.data_ptr(), int(max_candidates),
                   C.byref(best), C.byref(ms), _stream_ptr(stream))
        return {"tile": (best.tile_x, best.tile_y), "threads": best.block_threads,
                "ctas_per_sm": best.ctas_per_sm, "sweep_ms": ms.value}

    def roughness_async(self, heights, precision: int, out_buf, n_rows=10, n_cols=10, stream=None) -> None:
        ny, nx = heights.shape
        self._call("fsm_roughness", self.ptr, heights.data_ptr(), int(precision), nx, ny, int(n_rows),
                   int(n_cols), out_buf.data_ptr(), _stream_ptr(stream))

    def moment_partials(self, heights, about: float, stream=None) -> np.ndarray:
        """fsm_moment_partials of a CUDA height map: [n, sum d, min z, max z,
        sum |d|, sum d^2, sum d^3, sum d^4], d = z - about (host copy)."""
        import torch
        ny, nx = heights.shape
        prec = FSM_FP64 if heights.dtype == torch.float64 else FSM_FP32
        out = torch.zeros(8, dtype=torch.float64, device=heights.device)
        self._call("fsm_moment_partials", self.ptr, heights.data_ptr(), prec, nx, ny, float(about), out.data_ptr(),
                   _stream_ptr(stream))
        return out.cpu().numpy()

    def roughness(self, heights, n_rows=10, n_cols=10, stream=None) -> dict:
        import torch
        precision = FSM_FP64 if heights.dtype == torch.float64 else FSM_FP32
        buf = torch.zeros(ROUGH_BYTES, dtype=torch.uint8, device=heights.device)
        self.roughness_async(heights, precision, buf, n_rows, n_cols, stream)
        host = buf.cpu().numpy().tobytes()
        return rough_dict(RoughnessOut.from_buffer_copy(host))

    # -- batches ----------------------------------------------------------
    @staticmethod
    def _arrays(tools, procs, outs):
        n = len(outs)
        ta = (_P * n)(*[t.ptr for t in tools])
        pa = (_P * n)(*[p.ptr for p in procs])
        ha = (_P * n)(*[o.data_ptr() for o in outs])
        return n, ta, pa, ha

    def predict_batch(self, tools, procs, outs, rough_buf=None, tile=None, threads=None, counters=None,
                      stream=None, events=None, form=None, form_tasks=None) -> None:
        n, ta, pa, ha = self._arrays(tools, procs, outs)
        o = self._opts(tile, threads, counters, events, form=form, form_tasks=form_tasks)
        self._call("fsm_predict_batch", self.ptr, n, ta, pa, ha,
                   rough_buf.data_ptr() if rough_buf is not None else None,
                   C.byref(o) if o is not None else None, _stream_ptr(stream))

    def batch(self, tools, procs, outs, rough_buf=None, tile=None, threads=None, counters=None,
              events=None) -> "Batch":
        n, ta, pa, ha = self._arrays(tools, procs, outs)
        o = self._opts(tile, threads, counters, events)
        p = _P()
        self._call("fsm_batch_create", self.ptr, n, ta, pa, ha,
                   rough_buf.data_ptr() if rough_buf is not None else None,
                   C.byref(o) if o is not None else None, C.byref(p))
        return Batch(self, p.value)

    # -- server -----------------------------------------------------------
    def server_start(self, budget_bytes: int, n_streams: int = 4, max_batch: int = 256) -> None:
        self._call("fsm_server_start", self.ptr, int(budget_bytes), int(n_streams), int(max_batch))

    def server_stop(self) -> None:
        self._call("fsm_server_stop", self.ptr)

    def submit(self, tool: _Handle, proc: _Handle) -> int:
        t = C.c_uint64()
        self._call("fsm_submit", self.ptr, tool.ptr, proc.ptr, C.byref(t))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1) -> Optional[dict]:
        r = Result()
        rc = self._call("fsm_poll", self.ptr, C.c_uint64(ticket), int(timeout_ms), C.byref(r))
        if rc == FSM_PENDING:
            return None
        return {"d_heights": r.d_heights, "precision": r.precision, "nx": r.nx, "ny": r.ny,
                "rough": rough_dict(r.rough), "queue_s": r.queue_s, "latency_s": r.latency_s}

    def release(self, ticket: int) -> None:
        self._call("fsm_release_result", self.ptr, C.c_uint64(ticket))

    def cancel(self, ticket: int) -> None:
        self._call("fsm_cancel", self.ptr, C.c_uint64(ticket))

    def server_stats(self) -> dict:
        info = ServerInfo()
        self._call("fsm_server_stats", self.ptr, C.byref(info))
        return {k: getattr(info, k) for k, _ in ServerInfo._fields_ if k != "reserved"}

    def server_batches(self, capacity: int = 4096) -> List[dict]:
        buf = (BatchInterval * capacity)()
        n = C.c_int32()
        self._call("fsm_server_batches", self.ptr, buf, int(capacity), C.byref(n))
        return [{"slot": b.slot, "n_requests": b.n_requests, "t_start_ms": b.t_start_ms, "t_end_ms": b.t_end_ms}
                for b in buf[:n.value]]

    def server_inject_alloc_failures(self, count: int) -> None:
        self._call("fsm_server_inject_alloc_failures", self.ptr, int(count))


class Batch:
    """A prepared batch (fsm_batch_create); run() is graph-capturable."""

    def __init__(self, ctx: Context, ptr: int):
        self.ctx, self.ptr = ctx, ptr

    def run(self, stream=None) -> None:
        self.ctx._call("fsm_batch_run", self.ctx.ptr, self.ptr, _stream_ptr(stream))

    def close(self):
        if self.ptr:
            lib().fsm_batch_destroy(self.ctx.ptr, self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TRAJ_BYTES = 32  # sizeof(fsm_traj_point)


def trajectory_views(raw, n_teeth: int):
    """Views of a trajectory buffer: xyz [steps, n_teeth, 3] float64 and the
    edge index j and tooth [steps, n_teeth] int32."""
    import torch
    rec = raw.view(-1, TRAJ_BYTES)
    d = rec.view(-1).view(dtype=torch.float64).view(-1, 4)
    i = rec.view(-1).view(dtype=torch.int32).view(-1, 8)
    steps = rec.shape[0] // n_teeth
    return (d[:, :3].reshape(steps, n_teeth, 3), i[:, 6].reshape(steps, n_teeth),
            i[:, 7].reshape(steps, n_teeth))


def heights_tensor(proc: ProcessSpec, device="cuda"):
    import torch
    dt = torch.float64 if proc.precision == "fp64" else torch.float32
    return torch.empty((proc.ny, proc.nx), dtype=dt, device=device)


class _DeviceView:
    """__cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def result_view(res: dict):
    """A CUDA tensor viewing a served result's library-owned map (valid until
    release(ticket)); .clone() it to keep a copy."""
    import torch
    typestr = "<f8" if res["precision"] == FSM_FP64 else "<f4"
    return torch.as_tensor(_DeviceView(res["d_heights"], (res["ny"], res["nx"]), typestr), device="cuda")


def predict(workload: Workload, ctx: Optional[Context] = None, tile=None, counters=None):
    """One height map on the current CUDA device: returns a CUDA tensor."""
    ctx = ctx or Context(0)
    t, p = ctx.tool(workload.tool), ctx.process(workload.process)
    out = heights_tensor(workload.process)
    ctx.predict_surface(t, p, out, tile=tile, counters=counters)
    return out
