"""Helpers shared by the GPU tests: run the library and the oracle on the
same seeded workload and compare them with the stated tolerances."""
import numpy as np

# per-cell height tolerance (mm) against the FP64 oracle, and the share of
# cells allowed to differ because an edge point lies within 1e-12 mm of a
# sampling boundary (the oracle flags those cells)
TOL = {"fp64": 1e-9, "fp32": 5e-6}
SA_REL = {"fp64": 1e-9, "fp32": 1e-4}
MAX_TIE_FRACTION = 1e-4


def gpu_map(ctx, F, w, tile=None, counters=None, form=None, form_tasks=None):
    import torch
    t, p = ctx.tool(w.tool), ctx.process(w.process)
    out = F.heights_tensor(w.process)
    ctx.predict_surface(t, p, out, tile=tile, counters=counters, form=form, form_tasks=form_tasks)
    torch.cuda.synchronize()
    return out


def compare_maps(H_gpu, ref, prec):
    """Element-by-element comparison against the oracle result."""
    H = H_gpu.double().cpu().numpy() if hasattr(H_gpu, "cpu") else H_gpu
    ok = ~ref.flags
    assert ref.flags.mean() <= MAX_TIE_FRACTION, ref.flags.mean()
    err = np.abs(H - ref.H)
    worst = err[ok].max() if ok.any() else 0.0
    assert worst <= TOL[prec], "max |dz| = %.3e mm over %d cells" % (worst, int((err[ok] > TOL[prec]).sum()))
    return worst


def compare_roughness(r_gpu, r_ref, rel, keys=("Sa", "Sq")):
    for k in keys:
        a, b = r_gpu[k], r_ref[k]
        assert abs(a - b) <= rel * max(abs(b), 1e-300), (k, a, b)
