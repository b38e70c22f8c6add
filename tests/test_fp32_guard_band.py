"""The FP32 binning's guard band bounds its FP32 error (CPU, no GPU).

FP32 maps and the binning of FP64 maps place an edge point in a cell from
FP32 tile-local coordinates in cells; a point within the guard band of a
cell boundary is re-binned with the FP64 pose. The maps equal the FP64
binning only if the band bounds the FP32 error of every point. This test
models the sweep's FP32 arithmetic for the tile-local x and y of a pose --
the tool rows and the pass offsets divided by the pitch in float64 (the
rows' constant parts less half a cell, centring coordinates on cells) and
rounded once, the run anchor from a float pair of the pass offset and of the
feed per step (double-float affine step), fused multiply-adds of the rounded
phase table and tool rows -- with each fused multiply-add rounded once
(float32 products are exact in float64), against the same pose in float64,
over random tools, phases, tiles, pitches, feeds and run spans, and checks
the error in cells against the band the kernel computes for the run:
1.5 u (6 max(amp_x, amp_y) + 3 (|w_x| + |w_y| + |w_z|) + 3 tile pitch
+ 2 span) / pitch + 3 u tile + 1e-6, u = 2^-24."""
import numpy as np

U24 = 2.0 ** -24
f32 = np.float32


def fma32(a, b, c):
    """fmaf: a*b is exact in float64 for float32 a, b; one rounding to float32
    (the float64 sum's own rounding is far below float32's)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def two_sum(a, b):
    s = (a + b).astype(f32)
    bb = (s - a).astype(f32)
    e = ((a - (s - bb)) + (b - bb)).astype(f32)
    return s, e


def df_affine(d_hi, d_lo, n, f_hi, f_lo):
    """(d_hi + d_lo) + n (f_hi + f_lo) to float, the kernel's run anchor."""
    nf = n.astype(f32)
    p = (nf * f_hi).astype(f32)
    pe = fma32(nf, f_hi, -p)
    s, e = two_sum(d_hi, p)
    e = (e + ((d_lo + pe).astype(f32) + (nf * f_lo).astype(f32)).astype(f32)).astype(f32)
    return (s + e).astype(f32)


def test_guard_band_bounds_fp32_binning_error():
    rng = np.random.default_rng(20260328)
    worst = 0.0
    for pitch in (5e-4, 1e-3, 2e-3, 5e-3, 1e-2):
        for tile_x, tile_y in ((512, 76), (636, 61), (640, 34), (128, 32), (1024, 38)):
            n = 200_000
            amp = rng.uniform(0.0, 10.0, n)
            ax, ay = amp * rng.uniform(0.0, 1.0, n), amp * rng.uniform(0.0, 1.0, n)
            phx, phy = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)
            ux, vx, uy, vy = ax * np.cos(phx), ax * np.sin(phx), ay * np.cos(phy), ay * np.sin(phy)
            wx, wy, wz = rng.uniform(-10.0, 10.0, (3, n))
            th = rng.uniform(0.0, 2 * np.pi, n)
            c, s = np.cos(th), np.sin(th)
            fs = 10.0 ** rng.uniform(-5.0, -2.0, n)
            span = np.floor(rng.uniform(0.0, 1.0, n) * np.minimum(1e6, 20.0 / fs))  # steps of the run
            ds = np.floor(rng.uniform(0.0, 1.0, n) * (span + 1))                     # item's steps after the run start
            n_a = np.floor(rng.uniform(0.0, 1e6, n)).astype(np.int64)                 # pass step of the run start
            # tile-local targets near the tile, and the pass offset that puts the point there
            X = rng.uniform(-1.0, tile_x + 1.0, n) * pitch
            Y = rng.uniform(-1.0, tile_y + 1.0, n) * pitch
            px = c * ux + s * vx + wx
            d = X - ds * fs - px - n_a * fs          # pass_x0 - tile origin
            dyp = Y - (c * uy + s * vy + wy)         # pass line - tile origin (y)
            # FP32 inputs as the planner stores them: x and y rows in cells
            c32, s32 = c.astype(f32), s.astype(f32)
            # (the constant parts less half a cell: coordinates centred on cells)
            ux32, vx32, wx32 = (ux / pitch).astype(f32), (vx / pitch).astype(f32), (wx / pitch - 0.5).astype(f32)
            uy32, vy32, wy32 = (uy / pitch).astype(f32), (vy / pitch).astype(f32), (wy / pitch - 0.5).astype(f32)
            dc = d / pitch
            d_hi = dc.astype(f32)
            d_lo = (dc - d_hi.astype(np.float64)).astype(f32)
            fsc = fs / pitch
            fs_hi = fsc.astype(f32)
            fs_lo = (fsc - fs_hi.astype(np.float64)).astype(f32)
            # the kernel's FP32 arithmetic, in cells
            dxa = df_affine(d_hi, d_lo, n_a, fs_hi, fs_lo)
            fx = (fma32(ds.astype(f32), fs_hi, dxa) + fma32(c32, ux32, fma32(s32, vx32, wx32))).astype(f32)
            fy = ((dyp / pitch).astype(f32) + fma32(c32, uy32, fma32(s32, vy32, wy32))).astype(f32)
            # the same pose in float64 (the FP64 binning's coordinates, up to float64 rounding)
            ex = np.abs(fx.astype(np.float64) - (X / pitch - 0.5))
            ey = np.abs(fy.astype(np.float64) - (Y / pitch - 0.5))
            # the kernel's band for the run, in cells
            pt_err = 6.0 * np.maximum(ax, ay) + 3.0 * (np.abs(wx) + np.abs(wy) + np.abs(wz)) + \
                3.0 * max(tile_x, tile_y) * pitch
            g = 1.5 * U24 * (pt_err + 2.0 * span * fs) / pitch + 3.0 * U24 * max(tile_x, tile_y) + 1e-6
            ratio = np.maximum(ex, ey) / g
            assert ratio.max() < 1.0, (pitch, tile_x, tile_y, ratio.max())
            worst = max(worst, float(ratio.max()))
    # the band is a worst-case bound: the observed error stays well inside it
    assert worst < 0.7, worst


def test_guard_band_bounds_tilted_fp32_binning_error():
    """A feed direction phi off the X axis: the x and y rows are the feed
    frame's turned by phi (the band takes amp_a + amp_b for their
    amplitude), and y, like x, steps from its own run anchor: y = fma(ds,
    fsy, dyA) + fma(c, u_y, fma(s, v_y, w_y)) with dyA = the double-float
    affine step of the pass start's y, fsx = fs cos phi, fsy = fs sin phi."""
    rng = np.random.default_rng(20260329)
    worst = 0.0
    for pitch in (5e-4, 1e-3, 2e-3, 1e-2):
        for tile_x, tile_y in ((168, 170), (128, 135), (64, 64)):
            n = 200_000
            amp = rng.uniform(0.0, 10.0, n)
            aa, ab = amp * rng.uniform(0.0, 1.0, n), amp * rng.uniform(0.0, 1.0, n)
            pha, phb = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)
            ua, va, ub, vb = aa * np.cos(pha), aa * np.sin(pha), ab * np.cos(phb), ab * np.sin(phb)
            wa, wb, wz = rng.uniform(-10.0, 10.0, (3, n))
            phi = rng.uniform(0.0, 2 * np.pi, n)
            cf, sf = np.cos(phi), np.sin(phi)
            ux, uy = cf * ua - sf * ub, sf * ua + cf * ub
            vx, vy = cf * va - sf * vb, sf * va + cf * vb
            wx, wy = cf * wa - sf * wb, sf * wa + cf * wb
            th = rng.uniform(0.0, 2 * np.pi, n)
            c, s = np.cos(th), np.sin(th)
            fs = 10.0 ** rng.uniform(-5.0, -2.0, n)
            fsx, fsy = fs * cf, fs * sf
            span = np.floor(rng.uniform(0.0, 1.0, n) * np.minimum(1e6, 20.0 / fs))
            ds = np.floor(rng.uniform(0.0, 1.0, n) * (span + 1))
            n_a = np.floor(rng.uniform(0.0, 1e6, n)).astype(np.int64)
            X = rng.uniform(-1.0, tile_x + 1.0, n) * pitch
            Y = rng.uniform(-1.0, tile_y + 1.0, n) * pitch
            dx = X - ds * fsx - (c * ux + s * vx + wx) - n_a * fsx  # pass start - tile origin
            dy = Y - ds * fsy - (c * uy + s * vy + wy) - n_a * fsy
            c32, s32 = c.astype(f32), s.astype(f32)
            rows = [(r / pitch - h).astype(f32) for r, h in ((ux, 0), (vx, 0), (wx, 0.5), (uy, 0), (vy, 0), (wy, 0.5))]

            def pair(v):
                hi = v.astype(f32)
                return hi, (v - hi.astype(np.float64)).astype(f32)

            dx_hi, dx_lo = pair(dx / pitch)
            dy_hi, dy_lo = pair(dy / pitch)
            fx_hi, fx_lo = pair(fsx / pitch)
            fy_hi, fy_lo = pair(fsy / pitch)
            dxa = df_affine(dx_hi, dx_lo, n_a, fx_hi, fx_lo)
            dya = df_affine(dy_hi, dy_lo, n_a, fy_hi, fy_lo)
            ds32 = ds.astype(f32)
            fx = (fma32(ds32, (fsx / pitch).astype(f32), dxa) +
                  fma32(c32, rows[0], fma32(s32, rows[1], rows[2]))).astype(f32)
            fy = (fma32(ds32, (fsy / pitch).astype(f32), dya) +
                  fma32(c32, rows[3], fma32(s32, rows[4], rows[5]))).astype(f32)
            ex = np.abs(fx.astype(np.float64) - (X / pitch - 0.5))
            ey = np.abs(fy.astype(np.float64) - (Y / pitch - 0.5))
            pt_err = 6.0 * (aa + ab) + 3.0 * (np.abs(wx) + np.abs(wy) + np.abs(wz)) + \
                3.0 * max(tile_x, tile_y) * pitch
            g = 1.5 * U24 * (pt_err + 2.0 * span * fs) / pitch + 3.0 * U24 * max(tile_x, tile_y) + 1e-6
            ratio = np.maximum(ex, ey) / g
            assert ratio.max() < 1.0, (pitch, tile_x, tile_y, ratio.max())
            worst = max(worst, float(ratio.max()))
    assert worst < 0.7, worst
