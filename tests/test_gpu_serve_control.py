"""Request server: failure paths, cancellation, the table cache, device
overlap of batches, and the caller's current device.

Every failure here is made on the host (an injected allocation failure, a
request held back by the admission budget, a cancellation); no test faults,
traps or stalls the GPU. Results that complete must equal the same surface
predicted alone, bit for bit.
"""
import time

import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import Workload

pytestmark = pytest.mark.gpu

FSM_E_NOMEM, FSM_E_TIMEOUT, FSM_E_CANCELLED, FSM_E_STATE = -2, -4, -5, -6


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    ws = W.lhs_batch(n=6, seed=77, n_edge=40, rot_step_deg=0.5, side_range=(0.2, 0.4), pitch_range_um=(2.0, 4.0))
    alone = []
    for w in ws:
        alone.append(F.predict(w, ctx))
    torch.cuda.synchronize()
    return F, ctx, ws, alone


def test_poll_timeout_cancel_and_release(env):
    """The admission budget holds one 16 MB map but not two: a request
    submitted while a finished one still holds its map waits, a 1 ms poll of
    it times out, and releasing the first lets it run."""
    import torch
    F, ctx, ws, alone = env
    w = W.raster_ball_d10(precision="fp32", width=2.0, n_passes=2, n_edge=40, rot_step_deg=1.0)
    ref = F.predict(w, ctx)
    torch.cuda.synchronize()
    map_bytes = w.process.nx * w.process.ny * 4
    ctx.server_start(budget_bytes=int(1.5 * map_bytes), n_streams=2, max_batch=4)
    try:
        h = (ctx.tool(w.tool), ctx.process(w.process))
        a = ctx.submit(*h)
        ra = ctx.poll(a, timeout_ms=60000)  # done, but its map still holds the budget
        b = ctx.submit(*h)
        c = ctx.submit(*h)
        with pytest.raises(F.FsmError) as e:
            ctx.poll(b, timeout_ms=1)
        assert e.value.status == FSM_E_TIMEOUT
        assert ctx.poll(b, timeout_ms=0) is None  # FSM_PENDING: b carries on waiting
        # c is cancelled while queued: it never runs
        ctx.cancel(c)
        with pytest.raises(F.FsmError) as e:
            ctx.poll(c, timeout_ms=0)
        assert e.value.status == FSM_E_CANCELLED
        with pytest.raises(F.FsmError) as e:  # cancelling a finished request is a state error
            ctx.cancel(a)
        assert e.value.status == FSM_E_STATE
        assert torch.equal(F.result_view(ra), ref)
        ctx.release(a)  # frees the budget: b runs
        rb = ctx.poll(b, timeout_ms=60000)
        assert torch.equal(F.result_view(rb), ref)
        ctx.release(b)
        ctx.release(c)
        st = ctx.server_stats()
        assert st["cancelled"] == 1 and st["completed"] == 2 and st["queue_depth"] == 0
    finally:
        ctx.server_stop()


def test_injected_allocation_failure_then_recovery(env):
    import torch
    F, ctx, ws, alone = env
    ctx.server_start(budget_bytes=1 << 30, n_streams=2, max_batch=1)
    try:
        ctx.server_inject_alloc_failures(1)
        t = ctx.submit(ctx.tool(ws[1].tool), ctx.process(ws[1].process))
        with pytest.raises(F.FsmError) as e:
            ctx.poll(t, timeout_ms=60000)
        assert e.value.status == FSM_E_NOMEM
        ctx.release(t)
        st = ctx.server_stats()
        assert st["failed"] == 1 and st["bytes_in_use"] <= st["table_bytes"]
        # the server keeps serving
        tickets = [ctx.submit(ctx.tool(w.tool), ctx.process(w.process)) for w in ws]
        for tk, ref in zip(tickets, alone):
            r = ctx.poll(tk, timeout_ms=60000)
            assert torch.equal(F.result_view(r), ref)
            ctx.release(tk)
        st = ctx.server_stats()
        assert st["completed"] == len(ws) and st["failed"] == 1
    finally:
        ctx.server_stop()


def test_cancel_while_running_frees_the_map(env):
    F, ctx, ws, alone = env
    ctx.server_start(budget_bytes=1 << 30, n_streams=1, max_batch=8)
    try:
        tickets = [ctx.submit(ctx.tool(w.tool), ctx.process(w.process)) for w in ws]
        for tk in tickets:  # some are on the device, some still queued
            ctx.cancel(tk)
        for tk in tickets:
            with pytest.raises(F.FsmError) as e:
                ctx.poll(tk, timeout_ms=60000)
            assert e.value.status == FSM_E_CANCELLED
            ctx.release(tk)
        st = ctx.server_stats()
        assert st["cancelled"] == len(ws)
        assert st["bytes_in_use"] == st["table_bytes"]  # only cached tables remain
    finally:
        ctx.server_stop()


def test_table_cache_hits_give_the_same_surfaces(env):
    """Requests sharing a tool and set-up (ap, lead, tilt, step angle, phase)
    but not feed, step-over, grid or precision reuse the planned tables."""
    import torch
    F, ctx, ws, alone = env
    base = ws[2]
    variants = []
    for k, (fz_scale, prec) in enumerate([(1.0, "fp32"), (0.8, "fp32"), (1.3, "fp64"), (1.0, "fp64")]):
        p = base.process.replace(fz=base.process.fz * fz_scale, precision=prec, nx=base.process.nx - 7 * k)
        variants.append(Workload(base.name, base.tool, p))
    refs = [F.predict(v, ctx) for v in variants]
    torch.cuda.synchronize()
    ctx.server_start(budget_bytes=1 << 30, n_streams=2, max_batch=1)
    try:
        for rnd in range(2):
            for v, ref in zip(variants, refs):
                tk = ctx.submit(ctx.tool(v.tool), ctx.process(v.process))
                r = ctx.poll(tk, timeout_ms=60000)  # one at a time: each finds the tables of the last
                assert torch.equal(F.result_view(r), ref)
                ctx.release(tk)
        st = ctx.server_stats()
        assert st["table_misses"] == 1 and st["table_hits"] == 2 * len(variants) - 1, st
        assert st["tables_cached"] == 1
    finally:
        ctx.server_stop()


def test_batches_of_two_slots_overlap_on_the_device(env):
    """Requests arriving while a batch runs are launched on another slot's
    stream: the device-time intervals of batches on different slots
    intersect."""
    F, ctx, ws, alone = env
    many = W.lhs_batch(n=48, seed=78, n_edge=60, rot_step_deg=0.25, side_range=(0.5, 1.0),
                       pitch_range_um=(1.0, 2.0))
    ctx.server_start(budget_bytes=8 << 30, n_streams=3, max_batch=2)
    try:
        handles = [(ctx.tool(w.tool), ctx.process(w.process)) for w in many]
        tickets = []
        for h in handles:
            tickets.append(ctx.submit(*h))
            time.sleep(0.0005)
        for tk in tickets:
            ctx.poll(tk, timeout_ms=120000)
            ctx.release(tk)
        log = ctx.server_batches()
    finally:
        ctx.server_stop()
    assert sum(b["n_requests"] for b in log) == len(many)
    assert len({b["slot"] for b in log}) >= 2
    overlap = 0
    for i, a in enumerate(log):
        assert a["t_end_ms"] >= a["t_start_ms"] >= 0.0
        for b in log[i + 1:]:
            if a["slot"] != b["slot"] and a["t_start_ms"] < b["t_end_ms"] and b["t_start_ms"] < a["t_end_ms"]:
                overlap += 1
    assert overlap > 0, log


def _cudart():
    """The CUDA runtime libfsm.so is linked against (already loaded)."""
    import ctypes
    from paper_2603_28160_gb300 import fsm as F
    F.lib()
    for line in open("/proc/self/maps"):
        path = line.split()[-1]
        if "libcudart.so" in path:
            return ctypes.CDLL(path)
    pytest.skip("CUDA runtime not found in the process")


def test_entry_points_leave_the_current_device_alone(env):
    """Each entry point works on its context's device and gives the calling
    thread its previous current device back. With one GPU the check is that
    device 0 stays current; with two the caller sits on the other device."""
    import ctypes

    import torch
    F, ctx, ws, alone = env
    rt = _cudart()
    other = 1 if torch.cuda.device_count() > 1 else 0
    assert rt.cudaSetDevice(other) == 0
    w = ws[3]
    out = F.heights_tensor(w.process, device="cuda:0")
    ctx.predict_surface(ctx.tool(w.tool), ctx.process(w.process), out, stream=torch.cuda.Stream(device=0))
    dev = ctypes.c_int(-1)
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0 and dev.value == other
    ctx.server_start(budget_bytes=1 << 28, n_streams=1, max_batch=1)
    try:
        tk = ctx.submit(ctx.tool(w.tool), ctx.process(w.process))
        ctx.poll(tk, timeout_ms=60000)
        ctx.release(tk)
    finally:
        ctx.server_stop()
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0 and dev.value == other
    assert rt.cudaSetDevice(0) == 0
    torch.cuda.synchronize()
