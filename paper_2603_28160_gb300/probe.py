"""Binding of include/fsm_probe.h: measured rates of the GB300 units the
sweep and roughness kernels are bound by (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsm_probe.so")

FIELDS = ("fp32_flops", "fp64_flops", "f2i_ops", "i2f_ops", "frnd_ops", "int_ops", "lds_ops", "atoms32_ops",
          "atoms32_conf_ops", "atoms32_same_ops", "atoms64_ops")


class ProbeResult(C.Structure):
    _fields_ = [(f, C.c_double) for f in FIELDS] + [("sms", C.c_int32), ("reserved", C.c_int32),
                                                     ("ms_total", C.c_double)]


SIGNATURES = {"fsm_probe_run": [C.c_int, C.c_int, C.POINTER(ProbeResult)]}

_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfsm_probe.so is not built; run paper_2603_28160_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def run(device: int = 0, repeats: int = 3) -> dict:
    """All probes on `device`: rates in operations (flops for the FMA probes)
    per second over the whole GPU."""
    r = ProbeResult()
    rc = lib().fsm_probe_run(int(device), int(repeats), C.byref(r))
    if rc != 0:
        raise RuntimeError("fsm_probe_run failed with CUDA error %d" % rc)
    out = {f: getattr(r, f) for f in FIELDS}
    out["sms"] = r.sms
    out["ms_total"] = r.ms_total
    return out
