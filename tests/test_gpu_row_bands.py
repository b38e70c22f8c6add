"""One surface predicted in row bands (as ranks of several GPUs would, here
one after another on one GPU): each band map equals the rows of the whole
map, and the roughness combined from the bands' fsm_moment_partials equals
fsm_roughness of the whole map (Section 4.1.2 indicators)."""
import numpy as np
import pytest

from paper_2603_28160_gb300 import shard
from paper_2603_28160_gb300 import workloads as W
from paper_2603_28160_gb300.workloads import Workload

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_row_bands_rebuild_the_map_and_its_roughness(prec):
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    w = W.raster_ball_d10(precision=prec, width=0.6, pitch=0.002, n_passes=4, n_edge=60, rot_step_deg=0.5)
    full = F.predict(w, ctx)
    parts = []
    for k0, k1 in shard.row_bands(w.process.ny, 3):
        band = Workload(w.name, w.tool, shard.band_process(w.process, k0, k1))
        Hb = F.predict(band, ctx)
        torch.cuda.synchronize()
        if prec == "fp64":
            assert torch.equal(Hb, full[k0:k1])
        else:  # a point re-binned in FP64 in one tiling but not the other keeps its FP64 height, rounded
            assert (Hb - full[k0:k1]).abs().max().item() <= 1e-7
        parts.append(Hb)
    ref = ctx.roughness(full)

    def summed(about):
        v = [ctx.moment_partials(Hb, about) for Hb in parts]
        return [sum(x[0] for x in v), sum(x[1] for x in v), min(x[2] for x in v), max(x[3] for x in v),
                sum(x[4] for x in v), sum(x[5] for x in v), sum(x[6] for x in v), sum(x[7] for x in v)]

    first = summed(0.0)
    second = summed(0.0 + first[1] / first[0])
    got = shard.merge_moments(first, second, 0.0)
    for k in ("n", "zmin", "zmax"):
        assert got[k] == ref[k], k
    for k in ("mean", "Sz", "Sp", "Sv"):
        assert abs(got[k] - ref[k]) <= REL[prec] * max(abs(ref[k]), abs(ref["mean"])), (k, got[k], ref[k])
    for k in ("Sa", "Sq", "Ssk", "Sku"):
        assert abs(got[k] - ref[k]) <= 10 * REL[prec] * max(abs(ref[k]), 1e-300), (k, got[k], ref[k])


def test_moment_partials_against_numpy():
    import torch
    from paper_2603_28160_gb300 import fsm as F
    ctx = F.Context(0)
    rng = np.random.default_rng(12)
    for shape in [(1, 1), (3, 7), (257, 131), (700, 333)]:
        Hn = rng.normal(0.0, 0.002, size=shape) - 0.1
        for dt, rel in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            H = torch.from_numpy(Hn).to(dt).cuda()
            Hd = H.double().cpu().numpy()
            about = float(Hd.mean()) + 3e-4
            got = ctx.moment_partials(H, about)
            d = Hd - about
            want = [Hd.size, d.sum(), Hd.min(), Hd.max(), np.abs(d).sum(), (d * d).sum(), (d ** 3).sum(),
                    (d ** 4).sum()]
            assert got[0] == want[0] and got[2] == want[2] and got[3] == want[3]
            scale = [0, np.abs(d).sum(), 0, 0, np.abs(d).sum(), (d * d).sum(), (np.abs(d) ** 3).sum(),
                     (d ** 4).sum()]
            for k in (1, 4, 5, 6, 7):
                assert abs(got[k] - want[k]) <= rel * max(scale[k], 1e-300), (shape, dt, k, got[k], want[k])
