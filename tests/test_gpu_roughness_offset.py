"""Areal roughness (Section 3.2's Sa, Sq, Ssk, Sku about the mean plane) of
maps that sit far from zero -- a stock at 1000 mm or -250 mm with
micrometre texture -- against the FP64 oracle. FP32 maps sum their cells
about a reference cell (the map's first), so the FP32 leaves carry
deviations only and the error stays at the leaf bound whatever the offset;
FP64 maps sum the heights in FP64 (their mean is exact to FP64 rounding of
the mean itself)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("offset", [0.0, 1000.0, -250.0])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_roughness_far_from_zero(oracle_mod, offset, prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    rng = np.random.default_rng(11)
    dt = np.float32 if prec == "fp32" else np.float64
    Hn = (offset + rng.normal(0.0, 0.002, size=(777, 1301))).astype(dt)
    r = ctx.roughness(torch.from_numpy(Hn).cuda())
    ro = oracle_mod.roughness(Hn.astype(np.float64), 10, 10)
    rel = 2e-5 if prec == "fp32" else 1e-12
    # FP32: the mean to a small fraction of the texture, not of the offset;
    # FP64 sums the heights themselves, to FP64 rounding of the mean (each
    # FP64 deviation z - mu also carries half an ulp of the offset)
    tol = rel * ro["Sq"] if prec == "fp32" else 1e-13 * abs(ro["mean"]) + rel * ro["Sq"]
    assert abs(r["mean"] - ro["mean"]) <= tol, (r["mean"], ro["mean"])
    # a shift of the deviations by up to tol moves Sa and Sq by at most tol
    for k in ("Sa", "Sq"):
        assert abs(r[k] - ro[k]) <= rel * ro[k] + tol, (k, r[k], ro[k])
    assert r["zmin"] == ro["zmin"] and r["zmax"] == ro["zmax"]
    # Ssk and Sku move by about 3 and 4 (x Ssk) times dmu / Sq when the mean
    # moves by dmu: the mean's tolerance propagates into them
    for k in ("Ssk", "Sku"):
        bound = 100 * rel * max(abs(ro[k]), 1.0) + 4 * tol / ro["Sq"]
        assert abs(r[k] - ro[k]) <= bound, (k, r[k], ro[k])
