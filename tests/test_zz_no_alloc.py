"""fsm_roughness_noalloc: roughness for callers that may not allocate device
memory while they run (for example a host process that has already given all
device memory to its own pool, or a control loop with a fixed footprint). It
must return what fsm_roughness returns, call after call, using only the
library's fixed device array instead of fresh allocations."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCALARS = ("n", "mean", "zmin", "zmax", "Sa", "Sq", "Sp", "Sv", "Sz", "Ssk", "Sku")


def _roughness_via(ctx, F, entry_point, H, n_rows, n_cols):
    """Call one of the two C-ABI roughness entry points on a device map."""
    import torch
    precision = F.FSM_FP64 if H.dtype == torch.float64 else F.FSM_FP32
    out = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    ny, nx = H.shape
    ctx._call(entry_point, ctx.ptr, H.data_ptr(), precision, nx, ny, n_rows, n_cols, out.data_ptr(),
              F._stream_ptr(None))
    torch.cuda.synchronize()
    return F.rough_dict(F.RoughnessOut.from_buffer_copy(out.cpu().numpy().tobytes()))


def test_noalloc_matches_allocating_entry_point_two_calls_in_a_row():
    import torch

    from paper_2603_28160_gb300 import fsm as F
    from paper_2603_28160_gb300 import workloads as W

    ctx = F.Context(0)
    w = W.raster_ball_d10(precision="fp32", width=0.4, pitch=0.002, n_passes=4, n_edge=60, rot_step_deg=0.5)
    first = F.predict(w, ctx)  # an FP32 height map from the library
    rng = np.random.default_rng(7)
    second = torch.from_numpy(rng.normal(-0.1, 0.003, size=(333, 517))).cuda()  # FP64, another size
    for H, n_rows, n_cols in ((first, 10, 10), (second, 7, 13)):
        ref = _roughness_via(ctx, F, "fsm_roughness", H, n_rows, n_cols)
        got = _roughness_via(ctx, F, "fsm_roughness_noalloc", H, n_rows, n_cols)
        for k in SCALARS:
            assert abs(got[k] - ref[k]) <= 1e-12 * max(abs(ref[k]), 1e-300), (k, got[k], ref[k])
        assert got["row_index"] == ref["row_index"] and got["col_index"] == ref["col_index"]
        for k in ("Ra_row", "Rz_row", "Ra_col", "Rz_col"):
            assert np.allclose(got[k], ref[k], rtol=1e-12, atol=0.0, equal_nan=True), k


def _default_pool_attr(rt, attr, value=None):
    """Read (or, with value, set) a uint64 attribute of device 0's default
    stream-ordered memory pool, the pool fsm_roughness allocates from."""
    import ctypes
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), 0) == 0
    v = ctypes.c_uint64(0 if value is None else value)
    if value is None:
        assert rt.cudaMemPoolGetAttribute(pool, attr, ctypes.byref(v)) == 0
    else:
        assert rt.cudaMemPoolSetAttribute(pool, attr, ctypes.byref(v)) == 0
    return v.value


def test_noalloc_leaves_the_device_pool_untouched():
    """The defining property: no device allocation. The high watermark of
    the stream-ordered pool does not move across a no-alloc call, while the
    allocating entry point (the control) raises it."""
    import ctypes

    import torch

    from paper_2603_28160_gb300 import fsm as F

    USED_CURRENT, USED_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh
    ctx = F.Context(0)
    rt = None
    for line in open("/proc/self/maps"):
        if "libcudart.so" in line.split()[-1]:
            rt = ctypes.CDLL(line.split()[-1])
            break
    if rt is None:
        pytest.skip("CUDA runtime not found in the process")
    rng = np.random.default_rng(11)
    H = torch.from_numpy(rng.normal(0.0, 0.001, size=(700, 900)).astype(np.float32)).cuda()
    torch.cuda.synchronize()
    _roughness_via(ctx, F, "fsm_roughness_noalloc", H, 10, 10)  # first call: address look-up
    base = _default_pool_attr(rt, USED_CURRENT)
    _default_pool_attr(rt, USED_HIGH, 0)  # resets the watermark to what is in use now
    _roughness_via(ctx, F, "fsm_roughness_noalloc", H, 10, 10)
    _roughness_via(ctx, F, "fsm_roughness_noalloc", H, 10, 10)
    assert _default_pool_attr(rt, USED_HIGH) <= base
    _roughness_via(ctx, F, "fsm_roughness", H, 10, 10)  # control: allocates its partial sums
    assert _default_pool_attr(rt, USED_HIGH) > base


def test_noalloc_rejects_maps_above_its_limit():
    import torch

    from paper_2603_28160_gb300 import fsm as F

    ctx = F.Context(0)
    small = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(F.ROUGH_BYTES, dtype=torch.uint8, device="cuda")
    with pytest.raises(F.FsmError) as e:  # 2^15 x 2^15 cells: rejected on the host before any launch
        ctx._call("fsm_roughness_noalloc", ctx.ptr, small.data_ptr(), F.FSM_FP32, 1 << 15, 1 << 15, 10, 10,
                  out.data_ptr(), F._stream_ptr(None))
    assert e.value.status == -1 and "2^29" in str(e.value)
