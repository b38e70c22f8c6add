"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs, element by element, FP64 and FP32."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import ProcessSpec, ToolSpec, Workload

from .gpu_common import SA_REL, TOL, compare_maps, compare_roughness, gpu_map

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available()
    from paper_2603_28160_gb300 import fsm
    return fsm


@pytest.fixture(scope="module")
def ctx(F):
    return F.Context(0)


def with_prec(w, prec):
    return Workload(w.name, w.tool, w.process.replace(precision=prec))


SMALL = {
    "slot_flat_d6": lambda: W.slot_flat_d6(),
    "ball_raster_small": lambda: W.raster_ball_d10(width=0.5, pitch=0.002, n_passes=5, n_edge=80,
                                                   rot_step_deg=0.25),
    "ball_raster_ragged": lambda: W.raster_ball_d10(width=0.403, pitch=0.0013, n_passes=4, n_edge=50,
                                                    rot_step_deg=0.5),
    "floor_flat_d12_reduced": lambda: W.floor_flat_d12(width=0.5, pitch=0.002, rot_step_deg=2.0),
    # the paper's Case 2 face mill (round inserts, rake, per-insert runout), reduced patch
    "paper_case1_insert": lambda: W.paper_case(0, length=0.6, width=0.4, pitch=0.004, rot_step_deg=0.25,
                                               n_edge=60),
    "paper_case2_insert": lambda: W.paper_case(1, length=0.6, width=0.4, pitch=0.004, rot_step_deg=0.25,
                                               n_edge=60),
    "paper_case3_insert": lambda: W.paper_case(2, length=0.6, width=0.4, pitch=0.004, rot_step_deg=0.25,
                                               n_edge=60),
    # bull-nose end mill and zig-zag raster passes
    "torus_zigzag_lead": lambda: Workload("torus_zz", ToolSpec("torus", 8.0, 3, [30.0], n_edge=60, n_end=60,
                                                               corner_radius=1.5, runout_mm=0.004),
                                          ProcessSpec(fz=0.06, rpm=6000, rot_step_deg=0.5, ap=0.4, lead_deg=5.0,
                                                      pass_x0=-4.6, pass_y0=-0.9, steps_per_pass=8000, n_passes=4,
                                                      ae=0.6, x0=-0.3 + 0.31 * 0.004, y0=-0.3 + 0.37 * 0.004,
                                                      pitch=0.004, nx=150, ny=151, pass_mode="zigzag")),
    "ball_zigzag_tilt": lambda: Workload("ball_zz", ToolSpec("ball", 6.0, 2, [35.0], n_edge=70, runout_mm=0.006,
                                                             runout_phase_deg=70.0),
                                         ProcessSpec(fz=0.05, rpm=6000, rot_step_deg=0.5, ap=0.15, tilt_deg=8.0,
                                                     lead_deg=-4.0, pass_x0=-3.5, pass_y0=-0.25, steps_per_pass=36000,
                                                     n_passes=5, ae=0.12, x0=-0.25 + 0.31 * 0.003,
                                                     y0=-0.25 + 0.37 * 0.003, pitch=0.003, nx=167, ny=163,
                                                     pass_mode="zigzag", rot_sense=-1)),
    "flat_tilt_runout": lambda: Workload("flat_tilt", ToolSpec("flat", 3.0, 3, [35.0, 38.0, 41.0], n_edge=20,
                                                               n_end=80, runout_mm=0.008),
                                         ProcessSpec(fz=0.05, rpm=6000, rot_step_deg=1.0, ap=0.2, tilt_deg=4.0,
                                                     lead_deg=2.0, pass_x0=-2.6, pass_y0=-1.4,
                                                     steps_per_pass=8000, n_passes=3, ae=0.08,
                                                     x0=-0.1 + 0.31 * 0.003, y0=-0.1 + 0.37 * 0.003,
                                                     pitch=0.003, nx=67, ny=71)),
}


@pytest.mark.parametrize("name", sorted(SMALL))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_parity(ctx, F, oracle_mod, name, prec):
    import torch
    w = with_prec(SMALL[name](), prec)
    ref = oracle_mod.fsm(w, n_threads=8)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    H = gpu_map(ctx, F, w, counters=cnt)
    compare_maps(H, ref, prec)
    c = cnt.cpu().numpy()
    if prec == "fp64":
        assert c[1] == ref.stats["cutting"], (c, ref.stats)
    else:
        assert abs(int(c[1]) - ref.stats["cutting"]) <= 1e-5 * ref.stats["cutting"] + 2
    assert c[0] >= c[1]
    r = ctx.roughness(H)
    ro = oracle_mod.roughness(ref.H)
    if ro["Sq"] > 0:
        compare_roughness(r, ro, SA_REL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("tile", [(8, 8), (36, 20), (128, 32), (256, 64)])
def test_tiling_invariance(ctx, F, tile, prec):
    """Heights do not depend on the tile shape, bit for bit: a point's cell is
    its FP64 cell whether FP32 tile-local arithmetic or FP64 re-binning
    decided it, and its height is the map's own (FP64, or the FP32 pose's)
    either way."""
    w = with_prec(SMALL["ball_raster_ragged"](), prec)
    base = gpu_map(ctx, F, w).cpu().numpy()
    H = gpu_map(ctx, F, w, tile=tile).cpu().numpy()
    assert np.array_equal(H, base)


def test_roughness_against_oracle_random_maps(ctx, oracle_mod):
    import torch
    rng = np.random.default_rng(3)
    for shape in [(1, 1), (3, 7), (257, 131), (1000, 333)]:
        Hn = rng.normal(0.0, 0.002, size=shape) - 0.1
        # FP64 maps: FP64 throughout; FP32 maps: FP32 per-cell terms summed in
        # FP64 over 32-cell FP32 leaves (relative error ~1e-6)
        for dt, rel in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            H = torch.from_numpy(Hn).to(dt).cuda()
            n_rows, n_cols = min(10, shape[0]), min(10, shape[1])
            r = ctx.roughness(H, n_rows, n_cols)
            ro = oracle_mod.roughness(H.double().cpu().numpy(), n_rows, n_cols)
            for k in ("zmin", "zmax"):
                assert r[k] == ro[k], (shape, k)
            for k in ("mean", "Sa", "Sq"):
                assert abs(r[k] - ro[k]) <= rel * max(abs(ro[k]), 1e-300), (shape, k, r[k], ro[k])
            for k in ("Sp", "Sv", "Sz"):
                assert abs(r[k] - ro[k]) <= rel * max(abs(ro[k]), abs(ro["mean"])), (shape, k)
            if ro["Sq"] > 0:
                for k in ("Ssk", "Sku"):
                    assert abs(r[k] - ro[k]) <= 100 * rel * max(abs(ro[k]), 1.0), (shape, k)
            assert r["row_index"] == ro["row_index"] and r["col_index"] == ro["col_index"]
            for k in ("Ra_row", "Ra_col", "Rz_row", "Rz_col"):
                a, b = np.asarray(r[k]), np.asarray(ro[k])
                assert np.allclose(a, b, rtol=1e-12, atol=0, equal_nan=True), (shape, k)
