"""The oracle's multi-thread sweep equals its single-thread sweep bit for bit.

orc_fsm splits the global time steps into contiguous ranges, sweeps each
into a private map and merges the maps by minimum, the hit and boundary-tie
marks by union and the counts by sum. The per-cell minimum of Section 2.3 does
not depend on the order in which points arrive, so every thread count must
give the same map, the same tie flags and the same statistics as one thread.
The GPU parity tests compare against multi-thread oracle runs, so a merge
mistake (a dropped flag union, a count summed twice, a range boundary lost
between two threads) would otherwise go unnoticed.
"""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

THREADS = (2, 5, 12)


def _tie_workload():
    # the pass line lies exactly on a row boundary: the vertical ball tip is
    # a boundary tie at every step, so the tie flags are not empty
    tool = ToolSpec("ball", 4.0, 2, [0.0], n_edge=20)
    proc = ProcessSpec(fz=0.1, rpm=1000, rot_step_deg=1.0, ap=0.05, pass_x0=-2.5, pass_y0=0.0,
                       steps_per_pass=9000, x0=-0.1, y0=-0.1, pitch=0.005, nx=40, ny=40)
    return Workload("tie", tool, proc)


WORKLOADS = {
    # several passes, lead, runout: the ranges cut passes in the middle
    "ball_raster": lambda: W.raster_ball_d10(precision="fp64", width=0.3, pitch=0.002, n_passes=3, n_edge=40,
                                             rot_step_deg=1.0),
    # one pass with boundary ties
    "tie_single_pass": _tie_workload,
    # flat end, unequal helix, runout, bottom edge
    "flat_floor": lambda: W.floor_flat_d12(precision="fp64", width=0.3, pitch=0.004, rot_step_deg=4.0),
}


@pytest.fixture(scope="module", params=sorted(WORKLOADS))
def single(request, oracle_mod):
    w = WORKLOADS[request.param]()
    return w, oracle_mod.fsm(w, n_threads=1)


@pytest.mark.parametrize("k", THREADS)
def test_threads_equal_single_thread(single, oracle_mod, k):
    w, ref = single
    got = oracle_mod.fsm(w, n_threads=k)
    assert np.array_equal(got.H, ref.H)
    assert np.array_equal(got.flags, ref.flags)
    assert got.stats == ref.stats


def test_tie_workload_exercises_the_flag_union(oracle_mod):
    ref = oracle_mod.fsm(_tie_workload(), n_threads=1)
    assert ref.stats["cells_flagged"] > 0 and ref.flags.any()


def test_more_threads_than_steps(oracle_mod):
    """Thread counts above the number of time steps are clamped."""
    w = WORKLOADS["ball_raster"]()
    short = Workload(w.name, w.tool, w.process.replace(steps_per_pass=3, n_passes=2))
    ref = oracle_mod.fsm(short, n_threads=1)
    got = oracle_mod.fsm(short, n_threads=12)
    assert np.array_equal(got.H, ref.H) and got.stats == ref.stats
