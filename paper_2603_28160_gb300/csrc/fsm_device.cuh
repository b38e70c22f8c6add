// fsm_device.cuh -- device-side plan of one surface and the per-edge-point
// time-window enumeration of the tile sweep.
//
// Pose model (Section 2.1, Eq. eq_full_transformation, generalised to end
// mills with helix lag, axis runout and lead/tilt): edge point j of tooth K
// sits at q_Kj in the rotating tool frame; at global step s with spindle
// phase index m = s mod S and angle Theta_m = phase0 + sense * m * dtheta the
// point is at
//     w = c(s) + A Rz(Theta_m) q_Kj = c(s) + cos(Theta_m) u + sin(Theta_m) v + wq
// with u = A (qx, qy, 0), v = A (-qy, qx, 0), wq = qz A e_z, c(s) the tool
// reference point of the pass (Eq. eq_spindle_to_workpiece) and A the
// lead/tilt orientation. Each coordinate of w - c is a sinusoid in the step
// index: P_d(m) = wq_d + amp_d cos(dtheta (m - mph_d)). The sweep uses this
// to enumerate, for each tile, only the steps at which an edge point can
// fall inside the tile below the stock surface -- a per-point form of the
// tile's time window -- and evaluates each of those steps exactly.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define FSM_HD __host__ __device__ __forceinline__
#else
#define FSM_HD inline
#endif

#if !defined(__CUDACC__)
#include <math.h>
#endif

namespace fsm {

constexpr int kMaxTeeth = 16;
constexpr int kMaxArcs = 4;        // per edge point and pass after merging
constexpr float kMarginMm = 2e-5f; // enumeration slack in x, y, z (20 nm)
constexpr int kPlanParts = 256;    // max planning blocks per surface

// Per-surface plan. The host fills the inputs and table pointers; the plan
// kernel fills the derived block and the tables.
struct Surface {
    // ---- tool (inputs) ----
    int32_t kind, n_teeth, n_edge, n_end;
    double diameter, runout_mm, runout_phase_deg;
    double helix_deg[kMaxTeeth];
    double tooth_deg[kMaxTeeth];
    double insert_radius, rake_f_deg, rake_p_deg, eps_r_mm, eps_a_mm;
    double corner_radius;
    // ---- process (inputs) ----
    double fz, rot_step_deg, phase0_deg;
    int32_t rot_sense, n_passes;
    double ap, lead_deg, tilt_deg, ae, pass_x0, pass_y0;
    int32_t steps_per_pass, S;       // steps per pass, steps per revolution
    double stock_z, x0, y0, pitch;
    int32_t nx, ny, precision, E;    // E = points per tooth
    int32_t surface, pass_mode;      // FSM_SURFACE_*, FSM_PASS_*
    double wall_y;
    double feed_dir_deg;             // feed direction (degrees from +X)
    int32_t tilted;                  // feed_dir_deg is not a multiple of 360
    int32_t pad0;
    // ---- launch geometry (inputs) ----
    int32_t tile_x, tile_y, ntx, nty;
    int32_t form;             // FSM_FORM_* of the sweep's phase 2
    int32_t cached;           // tables and group bounds already built (a server's table cache)
    unsigned long long* form_tasks;  // NULL or [2]: tasks walked in the item / phase form
    // ---- tables (device pointers, inputs) ----
    // [N*E][4]: (ux,vx,wx,uz) (uy,vy,wy,vz) (wz,amp_y,mph_y,amp_z) (mph_z,amp_x,mph_x,0); the x and y
    // rows (ux..wy) are in cells (divided by the pitch; wx, wy less half a cell), everything else in mm
    float4* tool32;
    double* tool64;   // [9][N*E]: ux uy uz vx vy vz wx wy wz
    float2* ph32;     // [2S] (cos, sin) of Theta_m, m mod S: two turns, so m0 + offset needs no wrap
    double2* ph64;    // [2S]
    float4* groups;   // [N * ceil(E/32)]: (min P_y, max P_y while below the stock, min P_z, 0) over 32 points
    double* plan_part;  // [kPlanParts][4]: per planning block, lowest z, x and y reach
    int* tile_queue;    // next-tile counter of a single-surface sweep (zeroed by planning)
    void* heights;    // output map
    // ---- derived (plan kernel) ----
    // Map frame: the floor's is the workpiece frame; a wall's is (x, z, -y).
    // The tables hold map-frame vectors; the pass of pass index p runs at
    // map y = path_y0 + p * path_dy with map height offset z_ref, and the
    // un-machined surface sits at map height `stock`.
    double path_y0, path_dy, stock;
    double z_ref, fs, dtheta;       // map-frame reference height, feed per step, step angle (rad)
    double inv_pitch;               // 1 / pitch
    float reach_x, reach_y;         // max |P_x|, |P_y| over points and phases
    float zrel_f;                   // z_ref - stock
    float fs_hi, fs_lo;             // fs as an unevaluated float pair (fs_hi + fs_lo)
    float fs_f, inv_fs_f, dth_f, inv_dth_f, inv_pitch_f;
    float fsc_hi, fsc_lo, fsc_f;    // feed per step in cells (fs / pitch), as a float pair and rounded
    float pitch_f;                  // pitch (FP32 enumeration and error bounds)
    float guard_extra;              // FP32 rounding of the bin scaling, in cells
    // feed direction (tilted surfaces): the path of the +X process turned
    // about (pass_x0, pass_y0); pass p, position index k sits at
    // (pass_x0 + k fsx + p aex, pass_y0 + k fsy + p aey)
    double feed_c, feed_s;          // cos, sin of the feed direction
    double fsx, fsy, aex, aey;      // feed per step and step-over per pass, map x and y
    float feed_cf, feed_sf;
    float fscx_hi, fscx_lo, fscx_f; // fsx / pitch (cells per step) as a float pair and rounded
    float fscy_hi, fscy_lo, fscy_f; // fsy / pitch
};

// ---------------------------------------------------------------------------
// Order-preserving integer encoding of doubles: a < b <=> enc(a) < enc(b)
// as unsigned integers, so atomicMin on the encoding keeps the lowest height
// whatever order the edge points arrive in (FP64 cells; FP32 cells hold raw
// bits, see the sweep).
// ---------------------------------------------------------------------------
FSM_HD uint64_t enc64(uint64_t bits) {
    return (bits & 0x8000000000000000ull) ? ~bits : (bits | 0x8000000000000000ull);
}
FSM_HD uint64_t dec64(uint64_t e) {
    return (e & 0x8000000000000000ull) ? (e & 0x7fffffffffffffffull) : ~e;
}

// ---------------------------------------------------------------------------
// Arcs of spindle phase (in steps, on a circle of circumference S).
// ---------------------------------------------------------------------------
struct ArcF { float start, len; };           // real-valued, len in [0, S]
struct ArcI { int32_t m0, len; };             // integer phases m0 .. m0+len-1 (mod S)
struct Run { int32_t m0, len, s_lo, s_hi; };  // an ArcI restricted to steps [s_lo, s_hi]

// a mod S in [0, S) for the phase circle (exact enough for arc bookkeeping,
// which carries a step of slack).
FSM_HD float fmod_pos(float a, float S) {
    float r = a - S * floorf(a * (1.0f / S));
    if (r < 0.f) r += S;
    if (r >= S) r -= S;
    return r;
}

// a mod S in [0, S) for integers, through a float quotient corrected to exact.
FSM_HD int32_t imod_pos(int32_t a, int32_t S) {
    int32_t q = (int32_t)floorf((float)a * (1.0f / (float)S));
    int32_t r = a - q * S;
    while (r < 0) r += S;
    while (r >= S) r -= S;
    return r;
}

// floor(a / S) for a >= 0, through a float quotient corrected to exact.
FSM_HD int32_t idiv_floor(int32_t a, int32_t S) {
    int32_t q = (int32_t)((float)a * (1.0f / (float)S));
    while (q * S > a) --q;
    while ((q + 1) * S <= a) ++q;
    return q;
}

// cos of dth * d for a phase offset d (steps): reduced to [-pi, pi] first.
FSM_HD float phase_cos(float dth, float d, float S) {
    float r = fmod_pos(d, S);
    if (r > 0.5f * S) r -= S;
#if defined(__CUDA_ARCH__)
    return __cosf(dth * r);  // |error| < 4e-7 on [-pi, pi]; callers widen by 1e-5 relative
#else
    return cosf(dth * r);
#endif
}

// Phases where lo <= w + amp cos(dth (m - mph)) <= hi. Up to two arcs.
FSM_HD int band_arcs(float w, float amp, float mph, float lo, float hi, float inv_dth, float S,
                     ArcF* out) {
    if (!(amp > 1e-12f)) {
        if (w >= lo && w <= hi) { out[0].start = 0.f; out[0].len = S; return 1; }
        return 0;
    }
    float cl = (lo - w) / amp, ch = (hi - w) / amp;
    if (cl > 1.f || ch < -1.f || cl > ch) return 0;
    float a1 = ch >= 1.f ? 0.f : acosf(ch) * inv_dth;   // 0 .. S/2
    float a2 = cl <= -1.f ? 0.5f * S : acosf(cl) * inv_dth;
    if (a1 <= 0.f && a2 >= 0.5f * S) { out[0].start = 0.f; out[0].len = S; return 1; }
    if (a1 <= 0.f) { out[0].start = mph - a2; out[0].len = 2.f * a2; return 1; }
    if (a2 >= 0.5f * S) { out[0].start = mph + a1; out[0].len = S - 2.f * a1; return 1; }
    out[0].start = mph + a1; out[0].len = a2 - a1;
    out[1].start = mph - a2; out[1].len = a2 - a1;
    return 2;
}

// Phases where w + amp cos(dth (m - mph)) < hi. Zero or one arc.
FSM_HD int below_arc(float w, float amp, float mph, float hi, float inv_dth, float S, ArcF* out) {
    if (!(amp > 1e-12f)) {
        if (w < hi) { out->start = 0.f; out->len = S; return 1; }
        return 0;
    }
    float c0 = (hi - w) / amp;
    if (c0 > 1.f) { out->start = 0.f; out->len = S; return 1; }
    if (c0 <= -1.f) return 0;
    float b = acosf(c0) * inv_dth;
    out->start = mph + b;
    out->len = S - 2.f * b;
    return 1;
}

// Intersection of two arcs on the circle: up to two pieces.
FSM_HD int arc_intersect(ArcF a, ArcF b, float S, ArcF* out) {
    int n = 0;
    if (a.len >= S) { out[0] = b; return 1; }
    if (b.len >= S) { out[0] = a; return 1; }
    float d = fmod_pos(b.start - a.start, S);
    float lo = d > 0.f ? d : 0.f, hi = fminf(a.len, d + b.len);
    if (hi >= lo) { out[n].start = a.start + lo; out[n].len = hi - lo; ++n; }
    lo = 0.f; hi = fminf(a.len, d - S + b.len);
    if (hi >= lo) { out[n].start = a.start + lo; out[n].len = hi - lo; ++n; }
    return n;
}

// Widen real arcs to integer phase ranges (one step of slack on each side)
// and merge overlapping ones. Returns the number of merged arcs.
FSM_HD int to_int_arcs(const ArcF* in, int n, int32_t S, ArcI* out) {
    ArcI t[kMaxArcs];
    int k = 0;
    for (int a = 0; a < n; ++a) {
        int32_t m0 = (int32_t)floorf(in[a].start) - 1;
        int32_t m1 = (int32_t)ceilf(in[a].start + in[a].len) + 1;
        int32_t len = m1 - m0 + 1;
        if (len >= S) { out[0].m0 = 0; out[0].len = S; return 1; }
        t[k].m0 = imod_pos(m0, S);
        t[k].len = len;
        ++k;
    }
    // insertion sort by start
    for (int a = 1; a < k; ++a) {
        ArcI v = t[a];
        int b = a - 1;
        while (b >= 0 && t[b].m0 > v.m0) { t[b + 1] = t[b]; --b; }
        t[b + 1] = v;
    }
    int m = 0;
    for (int a = 0; a < k; ++a) {
        if (m > 0 && t[a].m0 <= out[m - 1].m0 + out[m - 1].len) {
            int32_t end = t[a].m0 + t[a].len;
            if (end > out[m - 1].m0 + out[m - 1].len) out[m - 1].len = end - out[m - 1].m0;
        } else {
            out[m++] = t[a];
        }
    }
    // wrap-around: the last arc may run past S into the first
    if (m > 1 && out[m - 1].m0 + out[m - 1].len >= out[0].m0 + S) {
        int32_t end = out[0].m0 + out[0].len + S;
        if (end > out[m - 1].m0 + out[m - 1].len) out[m - 1].len = end - out[m - 1].m0;
        for (int a = 0; a + 1 < m; ++a) out[a] = out[a + 1];
        --m;
    }
    for (int a = 0; a < m; ++a)
        if (out[a].len >= S) { out[0].m0 = 0; out[0].len = S; return 1; }
    return m;
}

// Range of w + amp cos(dth (m - mph)) over integer phases m0 .. m0+len-1.
FSM_HD void sinus_range(float w, float amp, float mph, ArcI a, float dth, int32_t S, float* lo,
                        float* hi) {
    if (a.len >= S || !(amp > 1e-12f)) {
        *lo = w - amp;
        *hi = w + amp;
        return;
    }
    float fS = (float)S;
    float e0 = phase_cos(dth, (float)a.m0 - mph, fS);
    float e1 = phase_cos(dth, (float)(a.m0 + a.len - 1) - mph, fS);
    float cmin = fminf(e0, e1), cmax = fmaxf(e0, e1);
    float span = (float)(a.len - 1);
    if (fmod_pos(mph - (float)a.m0, fS) <= span + 0.5f) cmax = 1.f;
    if (fmod_pos(mph + 0.5f * fS - (float)a.m0, fS) <= span + 0.5f) cmin = -1.f;
    *lo = w + amp * cmin;
    *hi = w + amp * cmax;
}

// Enumeration inputs of one edge point (FP32 table columns 2 and 3 plus wq).
struct PointGeom {
    float wx, wy, wz, amp_x, amp_y, amp_z, mph_x, mph_y, mph_z;
};

// t4: the point's FP32 table row; pitch: the map pitch (x and y rows are in
// cells, their constant parts less half a cell)
FSM_HD PointGeom load_geom(const float4* t4, float pitch) {
    PointGeom g;
    g.wx = (t4[0].z + 0.5f) * pitch;
    g.wy = (t4[1].z + 0.5f) * pitch;
    g.wz = t4[2].x;
    g.amp_y = t4[2].y;
    g.mph_y = t4[2].z;
    g.amp_z = t4[2].w;
    g.mph_z = t4[3].x;
    g.amp_x = t4[3].y;
    g.mph_x = t4[3].z;
    return g;
}

// A tilted surface's tables hold map-frame x, y rows but feed-frame
// sinusoids: turn the point's constant offset (map frame) into the feed
// frame (along, across the feed) with the direction's cos c and sin s.
FSM_HD void to_feed_frame(PointGeom& g, float c, float s) {
    const float a = c * g.wx + s * g.wy;
    const float b = c * g.wy - s * g.wx;
    g.wx = a;
    g.wy = b;
}

// Tile/pass frame for the enumeration, all in FP32 relative to the tile
// (a tilted surface's in the feed frame: x along the feed, y across it):
//   y band  [ylo, yhi]   of P_y (tile rows minus the pass's y, with margin)
//   z limit zhi          of P_z (stock - z_ref, with margin)
//   x:      pass step n lands P_x + dx0 + n*fs in [xlo, xhi]
struct TileFrame {
    float ylo, yhi, zhi;
    float xlo, xhi;     // tile x extent relative to the pass start, margin included
    float inv_fs;
    int32_t s0, n_steps;
    float inv_dth, dth;
    int32_t S;
    int32_t reversed;   // the pass runs back: step n sits at step n_steps-1-n
};

// All runs of one edge point for one (tile, pass): the steps at which it can
// land inside the tile below the stock. Returns the run count (<= kMaxArcs).
FSM_HD int point_runs(const PointGeom& g, const TileFrame& f, Run* runs) {
    const float fS = (float)f.S;
    ArcF ya[2], za[1], cut[kMaxArcs];
    int ny = band_arcs(g.wy, g.amp_y, g.mph_y, f.ylo, f.yhi, f.inv_dth, fS, ya);
    if (ny == 0) return 0;
    int nz = below_arc(g.wz, g.amp_z, g.mph_z, f.zhi, f.inv_dth, fS, za);
    if (nz == 0) return 0;
    int nc = 0;
    for (int a = 0; a < ny; ++a) nc += arc_intersect(ya[a], za[0], fS, cut + nc);
    if (nc == 0) return 0;
    ArcI ia[kMaxArcs];
    int ni = to_int_arcs(cut, nc, f.S, ia);
    int nr = 0;
    for (int a = 0; a < ni; ++a) {
        float pxlo, pxhi;
        sinus_range(g.wx, g.amp_x, g.mph_x, ia[a], f.dth, f.S, &pxlo, &pxhi);
        float slack = 1e-5f * g.amp_x + kMarginMm;
        // pass step n: xlo <= n*fs + P_x <= xhi
        float nlo = floorf((f.xlo - pxhi - slack) * f.inv_fs) - 1.f;
        float nhi = ceilf((f.xhi - pxlo + slack) * f.inv_fs) + 1.f;
        if (nlo < 0.f) nlo = 0.f;
        if (nhi > (float)(f.n_steps - 1)) nhi = (float)(f.n_steps - 1);
        if (nlo > nhi) continue;
        if (f.reversed) {  // the window was found for the mirrored step index
            const float lo2 = (float)(f.n_steps - 1) - nhi;
            nhi = (float)(f.n_steps - 1) - nlo;
            nlo = lo2;
        }
        runs[nr].m0 = ia[a].m0;
        runs[nr].len = ia[a].len;
        runs[nr].s_lo = f.s0 + (int32_t)nlo;
        runs[nr].s_hi = f.s0 + (int32_t)nhi;
        ++nr;
    }
    return nr;
}

// a + b as an unevaluated pair (hi, lo) with hi = fl(a + b) (Knuth's two-sum).
FSM_HD void two_sum(float a, float b, float* hi, float* lo) {
    const float s = a + b;
    const float bb = s - a;
    *lo = (a - (s - bb)) + (b - bb);
    *hi = s;
}

// (d_hi + d_lo) + n * (f_hi + f_lo) rounded to float, for an integer n that
// is exact in float (|n| < 2^24): the product's rounding error is recovered
// with an FMA, so the result is within about one rounding of the exact value.
FSM_HD float df_affine(float d_hi, float d_lo, int32_t n, float f_hi, float f_lo) {
    const float nf = (float)n;
    const float p = nf * f_hi;
    const float pe = fmaf(nf, f_hi, -p);
    float s, e;
    two_sum(d_hi, p, &s, &e);
    e += d_lo + pe + nf * f_lo;
    return s + e;
}

// Steps of a run: global steps s in [s_lo, s_hi] with (s - m0) mod S < len.
// occ0 is the first occurrence start (<= s_lo or the first after it),
// first/last segment lengths and the occurrence count give the total.
struct RunIter {
    int32_t occ0, first_off, len0, k_last, len_last, total;
};

FSM_HD RunIter run_iter(const Run& r, int32_t S) {
    RunIter it;
    int32_t base = r.s_lo - imod_pos(r.s_lo - r.m0, S);  // <= s_lo, == m0 mod S
    if (base + r.len - 1 < r.s_lo) base += S;
    it.occ0 = base;
    if (base > r.s_hi) { it.total = 0; it.len0 = 0; it.k_last = 0; it.len_last = 0; it.first_off = 0; return it; }
    int32_t f0 = base > r.s_lo ? base : r.s_lo;
    int32_t e0 = base + r.len - 1 < r.s_hi ? base + r.len - 1 : r.s_hi;
    it.first_off = f0 - base;
    it.len0 = e0 - f0 + 1;
    it.k_last = idiv_floor(r.s_hi - base, S);
    if (it.k_last == 0) {
        it.len_last = 0;
        it.total = it.len0;
    } else {
        int32_t ol = base + it.k_last * S;
        int32_t el = ol + r.len - 1 < r.s_hi ? ol + r.len - 1 : r.s_hi;
        it.len_last = el - ol + 1;
        it.total = it.len0 + (it.k_last - 1) * r.len + it.len_last;
    }
    return it;
}

}  // namespace fsm
