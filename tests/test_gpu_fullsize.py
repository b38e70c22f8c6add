"""Full-size parity: the 5x5 mm, 1 um ball-end raster (25 Mcells, 12 passes)
in the launch configuration bench.py times, every cell against the FP64 CPU
oracle, in FP64 and FP32, and every roughness indicator of the map (areal
and profile values) within a bound derived from the per-cell tolerance."""
import math

import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

from .gpu_common import SA_REL, TOL, compare_maps, compare_roughness, gpu_map

pytestmark = pytest.mark.gpu

# relative rounding of the roughness kernels' own sums (FP32 maps: FP32 terms
# over 32-cell leaves, double-float above; FP64 maps: FP64 throughout)
KERNEL_REL = {"fp64": 1e-12, "fp32": 2e-5}


def roughness_bounds(e, ro):
    """First-order bounds on the roughness differences of two maps whose
    cells differ by at most e (Section 4.1.2 definitions, mean plane = the
    arithmetic mean). With d = z - mean, every deviation moves by at most 2e
    (e from the cell, e from the mean), so:
        mean, zmin, zmax: e;  Sp, Sv, Sz, Sa, Sq, Ra, Rz: 2e;
        Ssk = <d^3>/Sq^3:  |d<d^3>| <= 3 <d^2> 2e = 6 e Sq^2, so
                           |dSsk| <= 6e/Sq + 3|Ssk| 2e/Sq = 6e (1 + |Ssk|)/Sq;
        Sku = <d^4>/Sq^4:  |d<d^4>| <= 4 <|d|^3> 2e <= 8e Sq^3 sqrt(Sku)
                           (Cauchy-Schwarz), so |dSku| <= 8e (sqrt(Sku) + Sku)/Sq.
    A factor 1.5 covers the second-order terms ((e/Sq)^2 ~ 1e-8 here)."""
    sq = ro["Sq"]
    b = {"mean": e, "zmin": e, "zmax": e, "Sp": 2 * e, "Sv": 2 * e, "Sz": 2 * e, "Sa": 2 * e, "Sq": 2 * e,
         "Ssk": 1.5 * 6 * e * (1 + abs(ro["Ssk"])) / sq,
         "Sku": 1.5 * 8 * e * (math.sqrt(ro["Sku"]) + ro["Sku"]) / sq}
    return b


@pytest.fixture(scope="module")
def reference(oracle_mod):
    import os
    w = W.raster_ball_d10(precision="fp64")
    return oracle_mod.fsm(w, n_threads=os.cpu_count() or 1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_fullsize_raster_ball(reference, oracle_mod, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w = W.raster_ball_d10(precision=prec)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, reference, prec)
    # this workload has no boundary ties, so every cell is within TOL and the
    # roughness bounds below hold for the whole map
    assert not reference.flags.any()
    Hn = H.double().cpu().numpy()
    e_cell = float(np.abs(Hn - reference.H).max())
    assert e_cell <= TOL[prec], e_cell
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == reference.stats["cutting"]
    else:
        assert abs(int(c[1]) - reference.stats["cutting"]) <= 1e-5 * reference.stats["cutting"] + 2
    r = ctx.roughness(H)
    ro = oracle_mod.roughness(reference.H)
    # the stated Sa/Sq targets (relative)
    compare_roughness(r, ro, SA_REL[prec], keys=("Sa", "Sq"))
    # every indicator within the bound the per-cell tolerance implies
    bounds = roughness_bounds(TOL[prec], ro)
    for k, b in bounds.items():
        lim = b + KERNEL_REL[prec] * abs(ro[k])
        assert abs(r[k] - ro[k]) <= lim, (k, r[k], ro[k], lim)
    # profiles along and across the feed (Ra, Rz: 2e each)
    assert r["row_index"] == ro["row_index"] and r["col_index"] == ro["col_index"]
    for k in ("Ra_row", "Rz_row", "Ra_col", "Rz_col"):
        a, b = np.asarray(r[k]), np.asarray(ro[k])
        lim = 2 * TOL[prec] + KERNEL_REL[prec] * np.abs(b)
        assert np.all(np.abs(a - b) <= lim), (k, a, b)
