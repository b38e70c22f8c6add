"""The paper's printed Case 2 parameters (tests/golden/paper_case2.json, with
citations) drive the insert workloads, and the paper's performance table is
consistent with a fixed time step (trajectory points x vc x fz constant)."""
import json
import math
import os

import pytest

from paper_2603_28160_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_case2.json")))


def test_insert_tool_matches_the_paper():
    t = GOLD["tool"]
    tool = W.paper_insert_tool()
    assert tool.kind == "insert" and tool.n_teeth == t["teeth"]
    assert tool.diameter == t["cutting_diameter_mm"]
    assert tool.insert_radius == t["corner_radius_mm"] == t["insert_diameter_mm"] / 2
    assert tool.rake_f_deg == t["radial_rake_deg"] and tool.rake_p_deg == t["axial_rake_deg"]


def test_cases_and_grid_match_the_paper():
    for (vc, fz, ap, er, ea), c, r in zip(W.PAPER_CASES, GOLD["conditions"]["rows"], GOLD["runout"]["rows"]):
        assert [vc, fz, ap] == c and [er, ea] == r
    assert [list(g) for g in W.PAPER_GRID] == [row[:3] for row in GOLD["performance"]["rows"]]
    w = W.paper_case(1)
    assert (w.process.fz, w.process.ap, w.tool.eps_r_mm, w.tool.eps_a_mm) == (0.4, 0.4, -0.026, 0.009)


def test_performance_table_implies_a_fixed_time_step():
    rows = GOLD["performance"]["rows"]
    for vc, fz, ap, pts, fsm_s, efsm_s, sp, sp10 in rows:
        assert pts * vc * fz == pytest.approx(15 * math.pi * 1e6, rel=2e-3)
        assert fsm_s / efsm_s == pytest.approx(sp, abs=0.15)  # printed speedups, truncated
    mean = sum(r[6] for r in rows) / len(rows)  # mean of the printed speedups
    assert mean == pytest.approx(GOLD["performance"]["mean_speedup"], abs=0.05)


def test_fixed_time_step_workload_reproduces_the_point_counts():
    """With a 0.2 us step and the tool centre travelling the 10 mm patch, the
    workload's time-step counts are the table's trajectory points (the printed
    counts for vc = 230 m/min differ by a few steps: 1e-5 relative)."""
    rows = GOLD["performance"]["rows"]
    for w, row in zip(W.paper_grid(dt_s=2e-7), rows):
        assert w.process.n_passes == 1
        assert abs(w.process.steps_per_pass - row[3]) <= 2e-5 * row[3], (w.name, w.process.steps_per_pass, row[3])
        spr = 360.0 / w.process.rot_step_deg
        assert abs(spr - round(spr)) < 1e-9
        rpm = 1000.0 * row[0] / (math.pi * 10.0)
        assert 60.0 / (rpm * round(spr)) == pytest.approx(2e-7, rel=1e-4)
