"""The sweep's per-point time windows cover every step that matters (CPU).

Phase 1 of the tile sweep (the per-tile restriction of Section 2.3's time
loop) never tests individual steps: for an edge point whose coordinates are
sinusoids of the spindle phase, P_d(m) = w_d + amp_d cos(dtheta (m - mph_d)),
it solves in FP32 for the arcs of phase where the point is inside the tile's
y band and below the stock, widens them by a step and a 20 nm margin, and
turns the tile's x extent into a window of pass steps. A step that puts the
point inside the tile below the stock but falls outside every run would be
silently lost. This test compiles the enumeration (the header the kernels
use, built for the host) and checks, against float64 brute force over every
step of the pass, that every such step lies in one of the returned runs --
for random geometries, phase counts, feeds, bands, stock levels and both
pass directions."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_28160_gb300", "csrc")


def cuda_include():
    """The CUDA headers next to nvcc (CUDA_HOME, then nvcc on the PATH)."""
    for root in (os.environ.get("CUDA_HOME"), os.path.dirname(os.path.dirname(shutil.which("nvcc") or "/x/x"))):
        if root and os.path.exists(os.path.join(root, "include", "cuda_runtime.h")):
            return os.path.join(root, "include")
    return None

SHIM = r"""
#include <cuda_runtime.h>
#include "fsm_device.cuh"
extern "C" int shim_point_runs(const float* g, const float* fr, const int* fi, int* out) {
    fsm::PointGeom geo;
    geo.wx = g[0]; geo.wy = g[1]; geo.wz = g[2];
    geo.amp_x = g[3]; geo.amp_y = g[4]; geo.amp_z = g[5];
    geo.mph_x = g[6]; geo.mph_y = g[7]; geo.mph_z = g[8];
    fsm::TileFrame f;
    f.ylo = fr[0]; f.yhi = fr[1]; f.zhi = fr[2]; f.xlo = fr[3]; f.xhi = fr[4];
    f.inv_fs = fr[5]; f.dth = fr[6]; f.inv_dth = fr[7];
    f.s0 = fi[0]; f.n_steps = fi[1]; f.S = fi[2]; f.reversed = fi[3];
    fsm::Run runs[fsm::kMaxArcs];
    const int n = fsm::point_runs(geo, f, runs);
    for (int a = 0; a < n; ++a) {
        out[4 * a] = runs[a].m0; out[4 * a + 1] = runs[a].len;
        out[4 * a + 2] = runs[a].s_lo; out[4 * a + 3] = runs[a].s_hi;
    }
    return n;
}
"""


@pytest.fixture(scope="module")
def shim():
    gxx, inc = shutil.which("g++"), cuda_include()
    if gxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    d = tempfile.mkdtemp()
    src, lib = os.path.join(d, "shim.cpp"), os.path.join(d, "shim.so")
    open(src, "w").write(SHIM)
    subprocess.check_call([gxx, "-O2", "-shared", "-fPIC", "-I", CSRC, "-I", inc, src, "-o", lib])
    L = C.CDLL(lib)
    L.shim_point_runs.restype = C.c_int
    yield L
    shutil.rmtree(d, ignore_errors=True)


def runs_of(L, g, fr, fi):
    out = (C.c_int * 16)()
    n = L.shim_point_runs((C.c_float * 9)(*g), (C.c_float * 8)(*fr), (C.c_int * 4)(*fi), out)
    return [tuple(out[4 * a:4 * a + 4]) for a in range(n)]


def test_runs_cover_every_step_inside_the_tile_below_the_stock(shim):
    rng = np.random.default_rng(28160)
    margin = 2e-5
    checked = 0
    for trial in range(4000):
        S = int(rng.choice([360, 720, 1440, 3600, 7200, 36000]))
        dth = 2.0 * np.pi / S
        w = rng.uniform(-3.0, 3.0, 3)
        amp = rng.uniform(0.0, 5.0, 3) * (rng.random(3) > 0.1)
        mph = rng.uniform(0.0, S, 3)
        fs = 10.0 ** rng.uniform(-4.0, -1.5)
        n_steps = int(rng.integers(200, 20000))
        s0 = int(rng.integers(0, 10**6))
        rev = int(rng.random() < 0.5)
        n = np.arange(n_steps)
        m = (s0 + n) % S
        P = [w[d] + amp[d] * np.cos(dth * (m - mph[d])) for d in range(3)]
        k = (n_steps - 1 - n) if rev else n
        x = k * fs + P[0]
        # a tile band and x window the point crosses, and a stock it dips below
        h = 10.0 ** rng.uniform(-3.0, -0.5)
        ya = rng.uniform(P[1].min() - h, P[1].max())
        wt = 10.0 ** rng.uniform(-2.5, 0.5)
        xa = rng.uniform(x.min() - wt, x.max())
        zz = rng.uniform(P[2].min(), P[2].max() + 0.1)
        inside = (P[1] >= ya) & (P[1] <= ya + h) & (x >= xa) & (x <= xa + wt) & (P[2] < zz)
        g = [w[0], w[1], w[2], amp[0], amp[1], amp[2], mph[0], mph[1], mph[2]]
        fr = [ya - margin, ya + h + margin, zz + margin, xa - margin, xa + wt + margin,
              np.float32(1.0 / fs), np.float32(dth), np.float32(1.0 / dth)]
        runs = runs_of(shim, g, fr, [s0, n_steps, S, rev])
        s = s0 + n[inside]
        covered = np.zeros(len(s), dtype=bool)
        for m0, ln, lo, hi in runs:
            covered |= (s >= lo) & (s <= hi) & (((s - m0) % S) < ln)
        assert covered.all(), (trial, int((~covered).sum()), runs)
        checked += len(s)
    assert checked > 5 * 10**4
