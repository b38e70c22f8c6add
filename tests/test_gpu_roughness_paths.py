"""FP32 roughness through both load paths of its passes against the FP64
oracle: a map that starts on a 16-byte boundary is read as float4 in leaves
of 8 per thread; one that does not (here: a view one float into its buffer)
cell by cell. Shapes cover a single cell, maps smaller than a float4, ragged
tails of every length mod 4, one chunk (32768 cells), one cell either side
of it, and maps of many chunks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 3), (2, 2), (1, 5), (3, 7), (181, 181), (128, 256), (32769, 1), (129, 255), (1000, 333),
          (2049, 1999)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2603_28160_gb300 import fsm as F
    return F.Context(0)


def check(r, ro, shape, rel=2e-5):
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


@pytest.mark.parametrize("shape", SHAPES)
def test_vector_and_scalar_paths_against_oracle(ctx, oracle_mod, shape):
    import torch
    rng = np.random.default_rng(shape[0] * 131 + shape[1])
    Hn = (rng.normal(0.0, 0.002, size=shape) - 0.1).astype(np.float32)
    n_rows, n_cols = min(10, shape[0]), min(10, shape[1])
    ro = oracle_mod.roughness(Hn.astype(np.float64), n_rows, n_cols)
    aligned = torch.from_numpy(Hn).cuda()
    assert aligned.data_ptr() % 16 == 0
    buf = torch.empty(Hn.size + 1, dtype=torch.float32, device="cuda")
    buf[1:] = aligned.reshape(-1)
    unaligned = buf[1:].view(shape)
    assert unaligned.data_ptr() % 16 == 4
    r_vec = ctx.roughness(aligned, n_rows, n_cols)
    r_cell = ctx.roughness(unaligned, n_rows, n_cols)
    check(r_vec, ro, shape)
    check(r_cell, ro, shape)
    # reproducible bit for bit
    r2 = ctx.roughness(aligned, n_rows, n_cols)
    for k in ("mean", "Sa", "Sq", "Ssk", "Sku", "zmin", "zmax"):
        assert r2[k] == r_vec[k] or (np.isnan(r2[k]) and np.isnan(r_vec[k])), k


def test_far_from_zero_and_constant(ctx, oracle_mod):
    """A map at 1000 mm with micrometre texture keeps its texture's precision
    (sums about the first cell), and a constant map gives Sq = 0 exactly."""
    import torch
    rng = np.random.default_rng(4)
    Hn = (1000.0 + rng.normal(0.0, 0.002, size=(513, 771))).astype(np.float32)
    r = ctx.roughness(torch.from_numpy(Hn).cuda())
    ro = oracle_mod.roughness(Hn.astype(np.float64), 10, 10)
    assert abs(r["mean"] - ro["mean"]) <= 2e-5 * ro["Sq"]
    for k in ("Sa", "Sq"):
        assert abs(r[k] - ro[k]) <= 2e-5 * ro[k] + 2e-5 * ro["Sq"], k
    Hc = np.full((300, 301), -0.25, np.float32)
    rc = ctx.roughness(torch.from_numpy(Hc).cuda())
    assert rc["mean"] == -0.25 and rc["Sq"] == 0.0 and rc["Sa"] == 0.0 and rc["Sz"] == 0.0
