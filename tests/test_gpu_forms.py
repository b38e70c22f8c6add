"""Both walks of the sweep's phase 2 against the oracle, on the same inputs.

The sweep evaluates the steps of a task's time window either step by step
(item form) or spindle phase by phase (phase form, which visits only the
revolutions of a phase that can reach the tile). The library chooses per task;
fsm_predict_opts.sweep_form forces one form and d_form_tasks reports which
form each task took. Each form, forced on its own, must give the oracle's map
(Section 2.3's per-cell minimum over exactly the points of Eq.
eq_sampling_boundaries), and the two forms must give the same map bit for bit:
they evaluate the same points with the same arithmetic.

Workloads are at their production discretisation (edge points and step
angle) on reduced windows: the ball raster of the benchmark, the flat-end
floor (300 flank + 6000 bottom points, 0.05 deg per step) and the flank's
side wall (1001 points, 0.05 deg per step), each over a short stretch of its
tool path so the oracle finishes in seconds.
"""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import Workload

from .gpu_common import compare_maps, gpu_map

pytestmark = pytest.mark.gpu


def _short_path(w, length_mm, n_passes=None, pass_y0=None):
    """Keep the tool and grid, run each pass over `length_mm` of feed centred
    on x = 0 (the map is the FSM output of that shorter path)."""
    p, t = w.process, w.tool
    S = round(360.0 / p.rot_step_deg)
    fs = t.n_teeth * p.fz / S
    steps = int(length_mm / fs)
    kw = dict(steps_per_pass=steps, pass_x0=-0.5 * steps * fs)
    if n_passes is not None:
        kw["n_passes"] = n_passes
    if pass_y0 is not None:
        kw["pass_y0"] = pass_y0
    return Workload(w.name + "_short", t, p.replace(**kw))


WORKLOADS = {
    # the benchmark's tool and discretisation (200 points, 0.1 deg) on 0.5 mm, 4 passes
    "ball_raster": lambda: W.raster_ball_d10(precision="fp64", width=0.5, n_passes=4),
    # the 20x20 mm floor's tool and discretisation on 0.4 mm; two passes 4.8 mm
    # apart straddle the window, the tool centre runs over 1 mm
    "floor_flat_d12": lambda: _short_path(W.floor_flat_d12(precision="fp64", width=0.4), 1.0, n_passes=2,
                                          pass_y0=-2.4),
    # the side wall's tool and discretisation on 0.4 mm of wall, 1 mm of path
    "side_wall_d12": lambda: _short_path(W.side_wall_flat_d12(precision="fp64", length=0.4), 1.0),
}


@pytest.fixture(scope="module")
def F():
    from paper_2603_28160_gb300 import fsm
    return fsm


@pytest.fixture(scope="module")
def ctx(F):
    return F.Context(0)


_REF = {}


def reference(oracle_mod, name):
    if name not in _REF:
        import os
        _REF[name] = oracle_mod.fsm(WORKLOADS[name](), n_threads=os.cpu_count() or 1)
    return _REF[name]


def _run(ctx, F, w, form):
    import torch
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    tasks = torch.zeros(2, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt, form=form, form_tasks=tasks)
    return H, cnt.cpu().numpy(), tasks.cpu().numpy()


@pytest.mark.parametrize("name", sorted(WORKLOADS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_forced_forms_match_oracle_and_each_other(ctx, F, oracle_mod, name, prec):
    base = WORKLOADS[name]()
    w = Workload(base.name, base.tool, base.process.replace(precision=prec))
    ref = reference(oracle_mod, name)
    maps = {}
    for form, slot in (("item", 0), ("phase", 1)):
        H, c, tasks = _run(ctx, F, w, form)
        assert tasks[slot] > 0 and tasks[1 - slot] == 0, (form, tasks)
        compare_maps(H, ref, prec)
        if prec == "fp64":
            assert c[1] == ref.stats["cutting"], (form, c, ref.stats)
        else:
            assert abs(int(c[1]) - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2
        maps[form] = (H.cpu().numpy(), c, int(tasks[slot]))
    assert np.array_equal(maps["item"][0], maps["phase"][0])
    assert maps["item"][1][1] == maps["phase"][1][1]  # same cutting count
    assert maps["item"][2] == maps["phase"][2]  # the same tasks, walked differently
    # the library's own choice gives the same map, whichever forms it took
    H, c, tasks = _run(ctx, F, w, "auto")
    assert int(tasks.sum()) == maps["item"][2]
    assert np.array_equal(H.cpu().numpy(), maps["item"][0])


def test_invalid_form_is_rejected(ctx, F):
    import torch
    w = W.raster_ball_d10(precision="fp32", width=0.05, n_passes=1, n_edge=8, rot_step_deg=1.0)
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    out = F.heights_tensor(w.process)
    o = F.PredictOpts()
    o.sweep_form = 7
    with pytest.raises(F.FsmError) as e:
        ctx._call("fsm_predict_surface", ctx.ptr, t.ptr, p.ptr, out.data_ptr(), F.C.byref(o), None)
    assert e.value.status == -1
    torch.cuda.synchronize()
