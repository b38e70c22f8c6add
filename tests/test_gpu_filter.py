"""ISO 16610-61 Gaussian S/L filtering on the GPU (fsm_filter) against the
FP64 oracle, element by element: random maps with ragged sizes and kernels
wider than the map, predicted maps, and sampled outputs of the full 25 Mcell
map with the paper's S-filter 10 um and L-filter 0.8 mm (Section 4.1.1).

Tolerances: FP64 maps 1e-9 mm per cell (double-float sums reach ~1e-14
relative); FP32 maps 5e-6 mm per cell against the oracle run on the same
float values (FP32 sums of up to 1601 products of heights below 0.3 mm)."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 5e-6}


def run_gpu(H, pitch, ls, lc):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    out = ctx.filter(torch.from_numpy(np.ascontiguousarray(H)).cuda(), pitch, ls, lc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [  # (ny, nx, pitch, lambda_s, lambda_c)
    (37, 53, 0.005, 0.0, 0.08),       # L only, kernel wider than the map
    (64, 700, 0.001, 0.0025, 0.04),   # S and L, rows longer than one block segment
    (301, 45, 0.002, 0.01, 0.0),      # S only, tall
    (129, 2400, 0.0005, 0.0012, 0.05),  # two segments per row plus a ragged third
    (17, 19, 0.01, 0.004, 0.006),     # lambda < pitch: one-tap filters
    (1, 333, 0.001, 0.0, 0.02),       # a single row
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_filter_random_maps(oracle_mod, case, prec):
    ny, nx, pitch, ls, lc = case
    rng = np.random.default_rng(nx * 7 + ny)
    H = -0.2 + 0.05 * rng.random((ny, nx)) + 0.01 * np.sin(np.arange(nx) * pitch / 0.03)[None, :]
    if prec == "fp32":
        H = H.astype(np.float32)
    got = run_gpu(H, pitch, ls, lc)
    ref = oracle_mod.sl_surface(H.astype(np.float64), pitch, ls, lc)
    assert got.dtype == H.dtype
    err = np.abs(got.astype(np.float64) - ref).max()
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_filter_predicted_map(oracle_mod, prec):
    """A predicted ball-raster map (1 x 1 mm at 2 um) through the paper's
    filters, then its roughness."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    from .gpu_common import gpu_map
    ctx = F.Context(0)
    w = W.raster_ball_d10(precision=prec, width=1.0, pitch=0.002, n_passes=5, n_edge=80, rot_step_deg=0.25)
    H = gpu_map(ctx, F, w)
    sl = ctx.filter(H, 0.002, 0.01, 0.8)
    torch.cuda.synchronize()
    ref = oracle_mod.sl_surface(H.double().cpu().numpy(), 0.002, 0.01, 0.8)
    assert np.abs(sl.double().cpu().numpy() - ref).max() <= TOL[prec]
    r = ctx.roughness(sl)
    ro = oracle_mod.roughness(ref)
    rel = 1e-9 if prec == "fp64" else 1e-4
    for k in ("Sa", "Sq"):
        assert abs(r[k] - ro[k]) <= rel * ro[k] + (0.0 if prec == "fp64" else 1e-9), (k, r[k], ro[k])


def test_filter_full_size_sampled(oracle_mod):
    """The 5 x 5 mm, 1 um map (25 Mcells, FP32 and FP64 as predicted), S 10 um
    and L 0.8 mm: outputs around an interior cell and a corner cell equal the
    oracle run on the part of the map they depend on (the S-filtered values
    within 800 um come from heights within 810 um)."""
    import torch
    from paper_2603_28160_gb300 import fsm as F
    from .gpu_common import gpu_map
    ctx = F.Context(0)
    pitch, ls, lc = 0.001, 0.010, 0.8
    reach = int(lc / pitch) + int(ls / pitch)
    for prec in ("fp32", "fp64"):
        w = W.raster_ball_d10(precision=prec)
        H = gpu_map(ctx, F, w)
        sl = ctx.filter(H, pitch, ls, lc)
        torch.cuda.synchronize()
        ny, nx = H.shape
        for (kc, ic) in ((2600, 2400), (3, 4)):
            k0, k1 = max(0, kc - reach - 4), min(ny, kc + reach + 5)
            i0, i1 = max(0, ic - reach - 4), min(nx, ic + reach + 5)
            ref = oracle_mod.sl_surface(H[k0:k1, i0:i1].double().cpu().numpy(), pitch, ls, lc)
            r0, r1, c0, c1 = max(kc - 4, 0), kc + 5, max(ic - 4, 0), ic + 5
            got = sl[r0:r1, c0:c1].double().cpu().numpy()
            exp = ref[r0 - k0:r1 - k0, c0 - i0:c1 - i0]
            assert got.shape == exp.shape == (r1 - r0, c1 - c0)
            assert np.abs(got - exp).max() <= TOL[prec], (prec, kc, ic, np.abs(got - exp).max())


def test_filter_rejects_bad_input():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    H = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(F.FsmError):
        ctx.filter(H, 0.001, 0.0, 5.0)    # lambda / pitch > 4096
    with pytest.raises(F.FsmError):
        ctx.filter(H, 0.0, 0.0, 0.1)
    with pytest.raises(F.FsmError):
        ctx.filter(H, 0.001, 0.0, 0.1, out=H)
