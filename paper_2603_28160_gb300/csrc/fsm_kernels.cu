// fsm_kernels.cu -- sm_103a kernels of the FSM surface generator.
//
//   plan_kernel      edge, phase and path tables of each surface in FP64
//                    (Section 2.2 discretisation; Section 3.2 "tool geometry"
//                    and "kinematics" modules precompute points and trig)
//   sweep_kernel<..> persistent tile sweep (Section 2.3 and the "surface
//                    computation module" of Section 3.2): a tile of the height
//                    map lives in shared memory, every edge point that can
//                    land in the tile below the stock is evaluated, binned by
//                    the sampling boundaries of Eq. eq_sampling_boundaries and
//                    folded in with a shared-memory atomic that keeps the
//                    lowest height (FP32 maps: signed atomicMax on the raw
//                    bits of a negative height; FP64 maps: atomicMin on an
//                    order-preserving integer encoding)
//   roughness        moments and profiles in a fixed reduction order, double-
//                    float sums on the FP32 pipes (Section 4.1.2)
//   trajectory       per step and tooth, the lowest edge point (Section 3.1)
#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <type_traits>

#include <mutex>

#include "fsm_device.cuh"
#include "fsm_host.h"
#include "fsm_internal.h"

namespace fsm {

// ===========================================================================
// Planning
// ===========================================================================
__device__ __forceinline__ double deg2rad(double d) { return d * (3.14159265358979323846 / 180.0); }

__device__ __forceinline__ double block_min_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmin(r, sh[w]);
    return r;
}
__device__ __forceinline__ float block_max_f(float v, float* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, sh[w]);
    return r;
}

// Tables of surface blockIdx.x; gridDim.y blocks share its edge points and
// phase entries. A single surface may arrive by value (`one`, graph-capture
// friendly); block (0,0) then stores it for the kernels that follow.
__global__ void __launch_bounds__(256) plan_kernel(Surface* surfs, int n, Surface one, int use_one) {
    const int sidx = blockIdx.x;
    if (sidx >= n) return;
    const Surface& sf = use_one ? one : surfs[sidx];
    if (use_one && blockIdx.y == 0 && threadIdx.x == 0) surfs[sidx] = one;
    if (sf.cached) return;  // tables built by an earlier launch and kept on the device
    __shared__ double A[9];
    __shared__ double kap[2];
    __shared__ double run_c[2];                  // runout offset (x, y)
    __shared__ double tooth_t[kMaxTeeth][2];     // per tooth: tan(helix), reference angle
    __shared__ double shd[32];
    __shared__ float shf[32];
    const int tid = threadIdx.x;
    const int N = sf.n_teeth, E = sf.E, S = sf.S;
    const double R = 0.5 * sf.diameter;
    const double sigma = (double)sf.rot_sense;
    const double dth = deg2rad(sf.rot_step_deg);
    // per-surface and per-tooth terms, once per block (blocks of at least 64 threads)
    if (tid < N) {
        tooth_t[tid][0] = tan(deg2rad(sf.helix_deg[tid]));
        tooth_t[tid][1] = -deg2rad(sf.tooth_deg[tid]);
    }
    __shared__ double ins[5];  // round insert: cos, sin of the radial rake; sin, cos of the axial rake; dL
    if (tid == 32) {
        const double lam = deg2rad(sf.runout_phase_deg);
        run_c[0] = sf.runout_mm * cos(lam);
        run_c[1] = sf.runout_mm * sin(lam);
    }
    if (tid == 33 && sf.kind == 2) {
        const double Ri = sf.insert_radius;
        const double gf = deg2rad(sf.rake_f_deg), gp = deg2rad(sf.rake_p_deg);
        // unfused products: R^2 - l^2 must be exactly 0 at l = +-R (an fma
        // would leave its rounding error there, possibly negative)
        const double rr = __dmul_rn(Ri, Ri);
        const double imm = Ri - sf.ap;
        const double dl_ap = sf.ap >= Ri ? Ri : sqrt(fmax(__dsub_rn(rr, __dmul_rn(imm, imm)), 0.0));
        const double dl_fz = sf.fz / (2.0 * cos(gf));
        ins[0] = cos(gf);
        ins[1] = sin(gf);
        ins[2] = sin(gp);
        ins[3] = cos(gp);
        ins[4] = fmin(fmax(dl_ap, dl_fz), Ri);
    }
    if (tid == 0) {
        double L = deg2rad(sf.lead_deg), T = deg2rad(sf.tilt_deg);
        double cL = cos(L), sL = sin(L), cT = cos(T), sT = sin(T);
        // A = Rx(-tilt) Ry(lead): the tool axis leans toward +X by lead, +Y by tilt
        A[0] = cL;        A[1] = 0.0; A[2] = sL;
        A[3] = -sT * sL;  A[4] = cT;  A[5] = sT * cL;
        A[6] = -cT * sL;  A[7] = -sT; A[8] = cT * cL;
        double tau = acos(fmin(1.0, A[8]));
        double c = fmin(1.0, fmax(-1.0, (R - sf.ap) / R));
        double half = acos(c);
        kap[0] = fmax(0.0, tau - half);
        kap[1] = fmin(0.5 * 3.14159265358979323846, tau + half);
        if (sf.surface == 1) {  // wall map frame (x, z, -y): rows (A0, A2, -A1)
            for (int k = 0; k < 3; ++k) {
                const double r1 = A[3 + k];
                A[3 + k] = A[6 + k];
                A[6 + k] = -r1;
            }
        }
    }
    __syncthreads();
    const int NE = N * E;
    const int first = blockIdx.y * blockDim.x + tid, stride = gridDim.y * blockDim.x;
    double zlo = 1e300;
    float rx = 0.f, ry = 0.f;
    for (int idx = first; idx < NE; idx += stride) {
        const int K = idx / E, j = idx - K * E;
        double qx, qy, qz;
        if (sf.kind == 2) {  // round insert: lower semicircle, rake, per-insert runout, tooth angle
            const double Ri = sf.insert_radius;
            const double rr = __dmul_rn(Ri, Ri);
            const double cgf = ins[0], sgf = ins[1], sgp = ins[2], cgp = ins[3], dL = ins[4];
            const double l = -dL + 2.0 * dL * ((double)j / (double)(E - 1));
            const double zc = Ri - sqrt(fmax(__dsub_rn(rr, __dmul_rn(l, l)), 0.0));
            // insert frame -> tool frame (x along the radius at the tooth's reference)
            const double xt = cgf * l + sgf * sgp * zc + R + (double)K * sf.eps_r_mm;
            const double yt = -sgf * l + cgf * sgp * zc;
            const double zt = cgp * zc + (double)K * sf.eps_a_mm;
            const double ta = tooth_t[K][1];
            qx = cos(ta) * xt - sin(ta) * yt + run_c[0];
            qy = sin(ta) * xt + cos(ta) * yt + run_c[1];
            qz = zt;
        } else {
            double r, h;
            if (sf.kind == 0) {  // flat: bottom edge then flank
                if (j < sf.n_end) {
                    r = R * ((double)j / (double)(sf.n_end - 1));
                    h = 0.0;
                } else {
                    r = R;
                    h = sf.ap * ((double)(j - sf.n_end) / (double)(sf.n_edge - 1));
                }
            } else if (sf.kind == 3) {  // torus: bottom flat, then the corner arc and flank by arc length
                const double rc = sf.corner_radius;
                if (j < sf.n_end) {
                    r = (R - rc) * ((double)j / (double)(sf.n_end - 1));
                    h = 0.0;
                } else {
                    const double arc_top = sf.ap >= rc ? 0.5 * 3.14159265358979323846 : acos(1.0 - sf.ap / rc);
                    const double len_arc = rc * arc_top;
                    const double len = len_arc + (sf.ap > rc ? sf.ap - rc : 0.0);
                    const double sa = len * ((double)(j - sf.n_end) / (double)(sf.n_edge - 1));
                    if (sa <= len_arc) {
                        const double kappa = sa / rc;
                        r = R - rc + rc * sin(kappa);
                        h = rc * (1.0 - cos(kappa));
                    } else {
                        r = R;
                        h = rc + (sa - len_arc);
                    }
                }
            } else {              // ball: uniform in polar angle over the engaged cap
                double kappa = kap[0] + (kap[1] - kap[0]) * ((double)j / (double)(E - 1));
                r = R * sin(kappa);
                h = R * (1.0 - cos(kappa));
            }
            const double psi = h * tooth_t[K][0] / R;  // helix lag
            const double alpha = tooth_t[K][1] - sigma * psi;
            double sa, ca;
            sincos(alpha, &sa, &ca);
            qx = r * ca + run_c[0];
            qy = r * sa + run_c[1];
            qz = h;
        }
        double u[3], v[3], w[3];
        for (int d = 0; d < 3; ++d) {
            u[d] = A[3 * d] * qx + A[3 * d + 1] * qy;
            v[d] = A[3 * d + 1] * qx - A[3 * d] * qy;
            w[d] = A[3 * d + 2] * qz;
        }
        float amp[3], mph[3];
        double a64[3];
#pragma unroll 1  // one copy of the FP64 sqrt/atan2/fmod code: it runs once, from a cold cache
        for (int d = 0; d < 3; ++d) {
            const double a = sqrt(u[d] * u[d] + v[d] * v[d]);
            a64[d] = a;
            double delta = atan2(v[d], u[d]);
            // Theta_m - delta = sense*dth*(m - mph)
            double m = sigma * (delta - deg2rad(sf.phase0_deg)) / dth;
            m = fmod(m, (double)S);
            if (m < 0.0) m += (double)S;
            amp[d] = (float)a;
            mph[d] = (float)m;
        }
        // lowest workpiece z of the point over a turn (exact FP64; min is
        // order-free): the map height on a floor, the map y on a wall; reach
        // along and across the feed
        const int dz = sf.surface == 1 ? 1 : 2;
        zlo = fmin(zlo, w[dz] - a64[dz]);
        rx = fmaxf(rx, (float)(fabs(w[0]) + a64[0]));
        ry = fmaxf(ry, (float)(fabs(w[1]) + a64[1]));
        // The sinusoids above are the feed frame's (the +X process); a
        // tilted surface's x and y rows are turned into the map frame.
        if (sf.tilted) {
            double fsn, fc;
            sincos(deg2rad(sf.feed_dir_deg), &fsn, &fc);
            double x = u[0], y = u[1];
            u[0] = fc * x - fsn * y;
            u[1] = fsn * x + fc * y;
            x = v[0];
            y = v[1];
            v[0] = fc * x - fsn * y;
            v[1] = fsn * x + fc * y;
            x = w[0];
            y = w[1];
            w[0] = fc * x - fsn * y;
            w[1] = fsn * x + fc * y;
        }
        double* t64 = sf.tool64;
        t64[0 * NE + idx] = u[0]; t64[1 * NE + idx] = u[1]; t64[2 * NE + idx] = u[2];
        t64[3 * NE + idx] = v[0]; t64[4 * NE + idx] = v[1]; t64[5 * NE + idx] = v[2];
        t64[6 * NE + idx] = w[0]; t64[7 * NE + idx] = w[1]; t64[8 * NE + idx] = w[2];
        // x and y rows in cells, so the sweep bins without a scaling step;
        // their constant parts less half a cell, so a point's tile-local
        // coordinate is centred on its cell: the nearest integer is the cell
        // and the remainder the signed distance from the cell's centre
        float4* t32 = sf.tool32 + 4 * (size_t)idx;
        const double ip = 1.0 / sf.pitch;
        t32[0] = make_float4((float)(u[0] * ip), (float)(v[0] * ip), (float)(w[0] * ip - 0.5), (float)u[2]);
        t32[1] = make_float4((float)(u[1] * ip), (float)(v[1] * ip), (float)(w[1] * ip - 0.5), (float)v[2]);
        t32[2] = make_float4((float)w[2], amp[1], mph[1], amp[2]);
        t32[3] = make_float4(mph[2], amp[0], mph[0], 0.f);
    }
    // phase table, two turns (entry m + S repeats entry m); its entries
    // continue the thread numbering after the edge points, so a grid sized
    // for both gives each thread one item (every residue mod stride is taken
    // by exactly one thread)
    int m_first = first - NE % stride;
    if (m_first < 0) m_first += stride;
    for (int m = m_first; m < S; m += stride) {
        double th = deg2rad(sf.phase0_deg + sigma * ((double)m * sf.rot_step_deg));
        double sn, cs;
        sincos(th, &sn, &cs);
        sf.ph64[m] = sf.ph64[m + S] = make_double2(cs, sn);
        sf.ph32[m] = sf.ph32[m + S] = make_float2((float)cs, (float)sn);
    }
    zlo = block_min_d(zlo, shd);
    rx = block_max_f(rx, shf);
    ry = block_max_f(ry, shf);
    if (tid == 0) {
        double* part = sf.plan_part + 4 * blockIdx.y;
        part[0] = zlo;
        part[1] = (double)rx;
        part[2] = (double)ry;
    }
}

// Reductions over the planning blocks, per-group bounds, derived scalars.
__global__ void __launch_bounds__(256) plan_finish_kernel(Surface* surfs, int n, int parts) {
    const int sidx = blockIdx.x;
    if (sidx >= n) return;
    Surface* sf = surfs + sidx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int N = sf->n_teeth, E = sf->E, S = sf->S;
    // the planning blocks' partials, reduced by the whole block (maxima as
    // minima of the negated values); cached tables keep the reduction of the
    // launch that built them in part 0
    __shared__ double shd[32];
    const int np = sf->cached ? 1 : parts;
    double zlo = 1e300, nrx = 0.0, nry = 0.0;
    for (int q = tid; q < np; q += blockDim.x) {
        zlo = fmin(zlo, sf->plan_part[4 * q]);
        nrx = fmin(nrx, -sf->plan_part[4 * q + 1]);
        nry = fmin(nry, -sf->plan_part[4 * q + 2]);
    }
    zlo = block_min_d(zlo, shd);
    const double rx = -block_min_d(nrx, shd), ry = -block_min_d(nry, shd);
    if (tid == 0) {
        if (sf->tile_queue) *sf->tile_queue = 0;
        if (!sf->cached) {
            sf->plan_part[0] = zlo;
            sf->plan_part[1] = rx;
            sf->plan_part[2] = ry;
        }
        const double dth = deg2rad(sf->rot_step_deg);
        double zr = sf->stock_z - sf->ap - zlo;  // workpiece height of the tool reference
        const double fs = (double)N * sf->fz / (double)S;
        if (sf->surface == 1) {  // wall: the pass runs at map y = its height, map z = -(its y)
            sf->path_y0 = zr;
            sf->path_dy = 0.0;
            sf->stock = -sf->wall_y;
            zr = -sf->pass_y0;
        } else {
            sf->path_y0 = sf->pass_y0;
            sf->path_dy = sf->ae;
            sf->stock = sf->stock_z;
        }
        sf->z_ref = zr;
        sf->fs = fs;
        sf->dtheta = dth;
        sf->inv_pitch = 1.0 / sf->pitch;
        sf->reach_x = (float)rx;
        sf->reach_y = (float)ry;
        sf->zrel_f = (float)(zr - sf->stock);
        sf->fs_hi = (float)fs;
        sf->fs_lo = (float)(fs - (double)sf->fs_hi);
        sf->fs_f = (float)fs;
        sf->inv_fs_f = (float)(1.0 / fs);
        sf->dth_f = (float)dth;
        sf->inv_dth_f = (float)(1.0 / dth);
        sf->inv_pitch_f = (float)(1.0 / sf->pitch);
        sf->pitch_f = (float)sf->pitch;
        const double fsc = fs / sf->pitch;
        sf->fsc_hi = (float)fsc;
        sf->fsc_lo = (float)(fsc - (double)sf->fsc_hi);
        sf->fsc_f = (float)fsc;
        double fsn = 0.0, fc = 1.0;
        if (sf->tilted) sincos(deg2rad(sf->feed_dir_deg), &fsn, &fc);
        sf->feed_c = fc;
        sf->feed_s = fsn;
        sf->feed_cf = (float)fc;
        sf->feed_sf = (float)fsn;
        sf->fsx = fs * fc;
        sf->fsy = fs * fsn;
        sf->aex = -sf->ae * fsn;
        sf->aey = sf->ae * fc;
        const double fcx = sf->fsx / sf->pitch, fcy = sf->fsy / sf->pitch;
        sf->fscx_hi = (float)fcx;
        sf->fscx_lo = (float)(fcx - (double)sf->fscx_hi);
        sf->fscx_f = (float)fcx;
        sf->fscy_hi = (float)fcy;
        sf->fscy_lo = (float)(fcy - (double)sf->fscy_hi);
        sf->fscy_f = (float)fcy;
        // the bin scaling x_l * (1/pitch) rounds twice, relative to |x_l / pitch|
        const double u24 = 5.9604644775390625e-8;
        sf->guard_extra = (float)(3.0 * u24 * (double)max(sf->tile_x, sf->tile_y) + 1e-6);
    }
    // per 32-point group bounds for the warp-level quick reject (warp per
    // group): the y range of the points over the phases in which they are
    // below the stock (the tile-independent z limit of the enumeration), and
    // their lowest z. A group outside a tile's y band has no runs there.
    // (Cached tables keep theirs: the limit, stock - z_ref, is ap plus the
    // tables' lowest z, a function of the cached inputs.) Warps 1.. take
    // the groups while warp 0 runs the scalar section above, so the scalars
    // they need are formed here by the same operations (launched with 256
    // threads: seven group warps).
    if (sf->cached || warp == 0) return;
    const double dth_l = deg2rad(sf->rot_step_deg);
    const double zr_l = sf->surface == 1 ? -sf->pass_y0 : sf->stock_z - sf->ap - zlo;
    const double stock_l = sf->surface == 1 ? -sf->wall_y : sf->stock_z;
    const float inv_dth_f = (float)(1.0 / dth_l), dth_f = (float)dth_l, pitch_f = (float)sf->pitch;
    double fsn_l = 0.0, fc_l = 1.0;
    if (sf->tilted) sincos(deg2rad(sf->feed_dir_deg), &fsn_l, &fc_l);
    const float feed_cf = (float)fc_l, feed_sf = (float)fsn_l;
    const int G = (E + 31) / 32;
    const float zhi = (float)(stock_l - zr_l) + kMarginMm;
    const float fS = (float)S;
    for (int gi = warp - 1; gi < N * G; gi += nw - 1) {
        const int K = gi / G, g = gi - K * G;
        const int j = g * 32 + lane;
        float ymin = 3.0e38f, ymax = -3.0e38f, zmin = 3.0e38f;
        if (j < E) {
            PointGeom geo = load_geom(sf->tool32 + 4 * (size_t)(K * E + j), pitch_f);
            if (sf->tilted) to_feed_frame(geo, feed_cf, feed_sf);
            zmin = geo.wz - geo.amp_z;
            ArcF za;
            ArcI ia[kMaxArcs];
            if (below_arc(geo.wz, geo.amp_z, geo.mph_z, zhi, inv_dth_f, fS, &za) > 0 &&
                to_int_arcs(&za, 1, S, ia) > 0) {
                sinus_range(geo.wy, geo.amp_y, geo.mph_y, ia[0], dth_f, S, &ymin, &ymax);
                const float slack = 1e-5f * geo.amp_y + kMarginMm;
                ymin -= slack;
                ymax += slack;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
            ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
            zmin = fminf(zmin, __shfl_xor_sync(0xffffffffu, zmin, o));
        }
        if (lane == 0) sf->groups[gi] = make_float4(ymin, ymax, zmin, 0.f);
    }
}

// ===========================================================================
// Tile sweep
// ===========================================================================
// Per-thread work counters. 32-bit per thread is enough (a thread handles
// well under 2^32 items of one launch); they are widened when flushed.
struct Counters {
    unsigned evaluated, cutting, rebinned, atomics;
};

__device__ __forceinline__ void warp_flush(Counters& c, long long* out) {
    if (out == nullptr) return;
    unsigned long long v[4] = {c.evaluated, c.cutting, c.rebinned, c.atomics};
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 4; ++k) atomicAdd((unsigned long long*)out + k, v[k]);
}

// A run of one edge point with its iteration bookkeeping (see run_iter).
struct RunRec {
    int32_t m0, len, occ0, first_off, len0;
    int32_t k_last, len_last;  // last revolution of the window and its length
    float dxA;      // FP32 path: tile-local x of the pass at the run's first step, in cells
    float g_cells;  // FP32 path: bin ambiguity band of this run (cells)
};

__device__ __forceinline__ int32_t rec_total(const RunRec& r) {
    return r.len0 + (r.k_last > 0 ? (r.k_last - 1) * r.len + r.len_last : 0);
}

constexpr int kRebinCap = 64;
// Mean revolutions per run phase from which a task takes the phase form of
// phase 2: 1.5 for FP32 maps (measured on the ball raster, ~1.7 on its
// feed-aligned tiles: 0.967 ms against 0.983 ms with a threshold of 3, which
// kept it item by item; floors and walls come back 4-20 times); 1.2 for
// FP64 maps, where the phase form also computes the FP64 height once per
// phase instead of once per item.
template <bool F64>
__device__ __forceinline__ bool phase_form_task(int items, int phases) {
    return F64 ? 5 * items >= 6 * phases : 2 * items >= 3 * phases;
}

// One warp's scratch: runs of 32 edge points and the FP64 re-binning queue.
// A point has up to kMaxArcs runs but rarely more than one (0.8 on
// average on the ball raster), so each lane keeps kRunSlots of them per
// round: a task whose points have more is walked in further rounds, each
// re-enumerating and keeping the next slots. The shared memory saved goes
// to the tile.
constexpr int kRunSlots = 2;
struct WarpScratch {
    RunRec run[32][kRunSlots];
    int32_t n[32];
    int32_t q_s[kRebinCap], q_m[kRebinCap], q_idx[kRebinCap];
    uint8_t flat[32 * kRunSlots];  // run list of the round: (point << 1) | slot
};

constexpr int kPassCache = 64;

// Per-tile values shared by all warps, computed once per tile in FP64.
// Tasks of a tile whose group-reject outcome is tabulated at the tile's
// start (one bit each; later tasks are tested as they are taken).
constexpr int kTaskBits = 4096;

struct TileShared {
    uint32_t accept[kTaskBits / 32];          // task t may have runs here (group reject passed)
    uint16_t acc_pre[kTaskBits / 32 + 1];     // accepted tasks in the words before word w
    float ylo[kPassCache], yhi[kPassCache];  // mm, for the enumeration (tilted: across the feed)
    float dy[kPassCache];                     // pass line - tile origin y, in cells (tilted: pass start y, hi)
    float dy_lo[kPassCache];                  // tilted: pass start y - tile origin y, lo part (cells)
    float dxp_hi[kPassCache], dxp_lo[kPassCache];  // tilted: pass start x - tile origin x (cells)
    uint8_t order[kPassCache];                // passes nearest the tile first (tasks are handed out in this order)
    float dx_hi, dx_lo;  // pass_x0 - tile origin x in cells, as a float pair
    float xlo, xhi;      // tile x extent relative to pass_x0, margins included (tilted: along the feed)
    float zhi;           // stock - z_ref + margin
};

// One pass seen from a tile: the enumeration's y band (mm; across the feed
// on a tilted surface) and the pass in tile-local cells -- its line's y on a
// +X feed; its start (x, y) as float pairs on a tilted feed.
struct PassFrame {
    float ylo, yhi;
    float dy;                   // +X feed: pass line y; tilted: start y (hi part)
    float dy_lo, dx_hi, dx_lo;  // tilted: start y (lo part), start x (pair)
};

template <typename Cell>
struct TileCtx {
    Cell* cells;          // [tile_y][tile_x] encodings
    int tx, ty;           // tile index
    int txc, tyc;         // valid cells in this tile
    double X0, Y0;        // tile origin (world)
};

struct Pose64 {
    double x, y, z;
};

struct Vec9 {
    double ux, uy, uz, vx, vy, vz, wx, wy, wz;
};

__device__ __forceinline__ Vec9 load_vec9(const double* t64, int NE, int idx) {
    Vec9 v;
    v.ux = t64[0 * NE + idx]; v.uy = t64[1 * NE + idx]; v.uz = t64[2 * NE + idx];
    v.vx = t64[3 * NE + idx]; v.vy = t64[4 * NE + idx]; v.vz = t64[5 * NE + idx];
    v.wx = t64[6 * NE + idx]; v.wy = t64[7 * NE + idx]; v.wz = t64[8 * NE + idx];
    return v;
}

// Every FP64 pose of the library (re-binning in the sweep, trajectory
// records) goes through these functions, with each rounding step spelled
// out, so a point is assigned to the same cell wherever it is re-binned.
__device__ __forceinline__ bool pass_reversed(const Surface& sf, int p) { return sf.pass_mode == 1 && (p & 1); }
// tool reference x, y at local step n of pass p (a zig-zag return pass runs
// back); a tilted surface's path is the +X path turned about (pass_x0, pass_y0)
__device__ __forceinline__ double path_x(const Surface& sf, int p, int32_t n) {
    const int32_t k = pass_reversed(sf, p) ? sf.steps_per_pass - 1 - n : n;
    if (sf.tilted) return __dadd_rn(sf.pass_x0, __fma_rn((double)k, sf.fsx, __dmul_rn((double)p, sf.aex)));
    return __dadd_rn(sf.pass_x0, __dmul_rn((double)k, sf.fs));
}
// the pass line's y on a +X feed
__device__ __forceinline__ double path_y(const Surface& sf, int p) {
    return __dadd_rn(sf.path_y0, __dmul_rn((double)p, sf.path_dy));
}
__device__ __forceinline__ double path_y(const Surface& sf, int p, int32_t n) {
    if (sf.tilted) {
        const int32_t k = pass_reversed(sf, p) ? sf.steps_per_pass - 1 - n : n;
        return __dadd_rn(sf.pass_y0, __fma_rn((double)k, sf.fsy, __dmul_rn((double)p, sf.aey)));
    }
    return path_y(sf, p);
}
// The z row takes the tool reference height into the point's constant first
// (w_z + z_ref), so the sweeps add it once per run and every FP64 height --
// sweep, re-bin, trajectory -- comes from the same three operations.
__device__ __forceinline__ Pose64 pose64(const Vec9& v, double2 cs, double xc, double yc, double zr) {
    Pose64 P;
    P.x = __dadd_rn(xc, __fma_rn(cs.x, v.ux, __fma_rn(cs.y, v.vx, v.wx)));
    P.y = __dadd_rn(yc, __fma_rn(cs.x, v.uy, __fma_rn(cs.y, v.vy, v.wy)));
    P.z = __fma_rn(cs.x, v.uz, __fma_rn(cs.y, v.vz, __dadd_rn(v.wz, zr)));
    return P;
}
__device__ __forceinline__ long long bin64(double coord, double origin, double inv_pitch) {
    return (long long)floor(__dmul_rn(__dsub_rn(coord, origin), inv_pitch));
}

// Tilted surfaces: the tile's extent along (a) and across (b) the feed,
// relative to (pass_x0, pass_y0), and the start of pass p in tile-local
// cells as float pairs.
template <typename Cell>
__device__ __forceinline__ void tile_feed_extent(const Surface& sf, const TileCtx<Cell>& tc, double* amin,
                                                 double* amax, double* bmin, double* bmax) {
    const double c = sf.feed_c, s = sf.feed_s;
    const double x0 = tc.X0 - sf.pass_x0, x1 = x0 + (double)tc.txc * sf.pitch;
    const double y0 = tc.Y0 - sf.pass_y0, y1 = y0 + (double)tc.tyc * sf.pitch;
    *amin = fmin(x0 * c, x1 * c) + fmin(y0 * s, y1 * s);
    *amax = fmax(x0 * c, x1 * c) + fmax(y0 * s, y1 * s);
    *bmin = fmin(y0 * c, y1 * c) - fmax(x0 * s, x1 * s);
    *bmax = fmax(y0 * c, y1 * c) - fmin(x0 * s, x1 * s);
}
template <typename Cell>
__device__ __forceinline__ void pass_start_cells(const Surface& sf, const TileCtx<Cell>& tc, int p, float* dx_hi,
                                                 float* dx_lo, float* dy_hi, float* dy_lo) {
    const double dx = (__dadd_rn(sf.pass_x0, __dmul_rn((double)p, sf.aex)) - tc.X0) * sf.inv_pitch;
    const double dy = (__dadd_rn(sf.pass_y0, __dmul_rn((double)p, sf.aey)) - tc.Y0) * sf.inv_pitch;
    *dx_hi = (float)dx;
    *dx_lo = (float)(dx - (double)*dx_hi);
    *dy_hi = (float)dy;
    *dy_lo = (float)(dy - (double)*dy_hi);
}

template <bool kTilt, typename Cell>
__device__ __forceinline__ void fill_tile_shared(const Surface& sf, const TileCtx<Cell>& tc, TileShared& ts) {
    const int np = min(sf.n_passes, kPassCache);
    if (kTilt && sf.tilted) {
        double amin, amax, bmin, bmax;
        tile_feed_extent(sf, tc, &amin, &amax, &bmin, &bmax);
        for (int p = threadIdx.x; p < np; p += blockDim.x) {
            ts.ylo[p] = (float)(bmin - (double)p * sf.ae) - kMarginMm;
            ts.yhi[p] = (float)(bmax - (double)p * sf.ae) + kMarginMm;
            pass_start_cells(sf, tc, p, &ts.dxp_hi[p], &ts.dxp_lo[p], &ts.dy[p], &ts.dy_lo[p]);
        }
        if (threadIdx.x == 0) {
            ts.dx_hi = ts.dx_lo = 0.f;
            ts.xlo = (float)amin - kMarginMm;
            ts.xhi = (float)amax + kMarginMm;
            ts.zhi = (float)(sf.stock - sf.z_ref) + kMarginMm;
        }
        return;
    }
    const double y1 = tc.Y0 + (double)tc.tyc * sf.pitch;
    for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const double yc = path_y(sf, p);
        ts.ylo[p] = (float)(tc.Y0 - yc) - kMarginMm;
        ts.yhi[p] = (float)(y1 - yc) + kMarginMm;
        ts.dy[p] = (float)((yc - tc.Y0) * sf.inv_pitch);
    }
    if (threadIdx.x == 0) {
        const double d = (sf.pass_x0 - tc.X0) * sf.inv_pitch;
        ts.dx_hi = (float)d;
        ts.dx_lo = (float)(d - (double)ts.dx_hi);
        ts.xlo = (float)(tc.X0 - sf.pass_x0) - kMarginMm;
        ts.xhi = (float)(tc.X0 + (double)tc.txc * sf.pitch - sf.pass_x0) + kMarginMm;
        ts.zhi = (float)(sf.stock - sf.z_ref) + kMarginMm;
    }
}

// y band of pass p relative to the pass line, and the pass relative to the tile
template <bool kTilt, typename Cell>
__device__ __forceinline__ void pass_band(const Surface& sf, const TileCtx<Cell>& tc, const TileShared& ts,
                                          int p, PassFrame& pf) {
    if (p < kPassCache) {
        pf.ylo = ts.ylo[p];
        pf.yhi = ts.yhi[p];
        pf.dy = ts.dy[p];
        if (kTilt && sf.tilted) {
            pf.dy_lo = ts.dy_lo[p];
            pf.dx_hi = ts.dxp_hi[p];
            pf.dx_lo = ts.dxp_lo[p];
        }
    } else if (kTilt && sf.tilted) {
        double amin, amax, bmin, bmax;
        tile_feed_extent(sf, tc, &amin, &amax, &bmin, &bmax);
        pf.ylo = (float)(bmin - (double)p * sf.ae) - kMarginMm;
        pf.yhi = (float)(bmax - (double)p * sf.ae) + kMarginMm;
        pass_start_cells(sf, tc, p, &pf.dx_hi, &pf.dx_lo, &pf.dy, &pf.dy_lo);
    } else {
        const double yc = path_y(sf, p);
        pf.ylo = (float)(tc.Y0 - yc) - kMarginMm;
        pf.yhi = (float)(tc.Y0 + (double)tc.tyc * sf.pitch - yc) + kMarginMm;
        pf.dy = (float)((yc - tc.Y0) * sf.inv_pitch);
    }
}

// Phase 1 of a warp task: lane = edge point j = 32 g + lane of tooth K. Each
// lane enumerates its runs for pass p and stores those of round `round`
// (its runs kRunSlots round .. kRunSlots (round + 1) - 1) with their
// iteration bookkeeping, FP32 anchor and guard band. t4 and zb (the FP32
// height base z_ref - stock + w_z) stay in the lane's registers for phase 2.
// Returns whether any lane has work this round; *more: some lane has runs
// beyond it.
template <bool kTilt>
__device__ __forceinline__ bool warp_runs(const Surface& sf, const TileShared& ts, const PassFrame& pf, int K,
                                          int g, int p, WarpScratch& ws, float4 (&t4)[3], float& zb, int round,
                                          bool* more, int* items, int* phases) {
    const int lane = threadIdx.x & 31;
    const int E = sf.E;
    const int j = g * 32 + lane;
    const int v0 = kRunSlots * round;  // this round's first run index
    int nr = 0, nv = 0;                 // runs kept this round, valid runs of the point
    t4[0] = t4[1] = t4[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    zb = 0.f;
    if (j < E) {
        const float4* tp = sf.tool32 + 4 * (size_t)(K * E + j);
        t4[0] = tp[0];
        t4[1] = tp[1];
        t4[2] = tp[2];
        const float4 t3 = tp[3];
        PointGeom geo;
        const float pitch = sf.pitch_f;  // the x, y rows are in cells
        geo.wx = (t4[0].z + 0.5f) * pitch;
        geo.wy = (t4[1].z + 0.5f) * pitch;
        geo.wz = t4[2].x;
        geo.amp_y = t4[2].y;
        geo.mph_y = t4[2].z;
        geo.amp_z = t4[2].w;
        geo.mph_z = t3.x;
        geo.amp_x = t3.y;
        geo.mph_x = t3.z;
        // FP32 error bounds of z and of the tile-local x, y for this point
        // (error model in the precision-scheme documentation), 1.5x margin;
        // on a tilted surface the map-frame x and y sinusoids are mixtures
        // of the tabulated feed-frame ones (amplitude at most their sum)
        const float u24 = 5.9604644775390625e-8f;
        const bool tilted = kTilt && sf.tilted;
        const float amp_xy = tilted ? geo.amp_x + geo.amp_y : fmaxf(geo.amp_x, geo.amp_y);
        const float pt_err = 6.f * amp_xy + 3.f * (fabsf(geo.wx) + fabsf(geo.wy) + fabsf(geo.wz)) +
                             3.f * (float)max(sf.tile_x, sf.tile_y) * pitch;
        if (tilted) to_feed_frame(geo, sf.feed_cf, sf.feed_sf);
        TileFrame f;
        f.ylo = pf.ylo;
        f.yhi = pf.yhi;
        f.zhi = ts.zhi;
        f.xlo = ts.xlo;
        f.xhi = ts.xhi;
        f.inv_fs = sf.inv_fs_f;
        f.s0 = p * sf.steps_per_pass;
        f.n_steps = sf.steps_per_pass;
        f.dth = sf.dth_f;
        f.inv_dth = sf.inv_dth_f;
        f.S = sf.S;
        f.reversed = pass_reversed(sf, p) ? 1 : 0;
        Run runs[kMaxArcs];
        const int n = point_runs(geo, f, runs);
        zb = sf.zrel_f + geo.wz;
        for (int a = 0; a < n; ++a) {
            const RunIter it = run_iter(runs[a], sf.S);
            if (it.total <= 0) continue;
            const int v = nv++;
            *items += it.total;  // (all of the point's runs, whichever round keeps them)
            *phases += runs[a].len;
            if (v < v0 || v >= v0 + kRunSlots) continue;
            RunRec& r = ws.run[lane][nr++];
            r.m0 = runs[a].m0;
            r.len = runs[a].len;
            r.occ0 = it.occ0;
            r.first_off = it.first_off;
            r.len0 = it.len0;
            r.k_last = it.k_last;
            r.len_last = it.len_last;
            const int32_t sA = it.occ0 + it.first_off;
            const int32_t nA = f.reversed ? f.n_steps - 1 - (sA - f.s0) : sA - f.s0;
            if (tilted)
                r.dxA = df_affine(pf.dx_hi, pf.dx_lo, nA, sf.fscx_hi, sf.fscx_lo);  // cells
            else
                r.dxA = df_affine(ts.dx_hi, ts.dx_lo, nA, sf.fsc_hi, sf.fsc_lo);  // cells
            const float span_mm = (float)(runs[a].s_hi - runs[a].s_lo) * sf.fs_f;
            r.g_cells = 1.5f * u24 * (pt_err + 2.f * span_mm) * sf.inv_pitch_f + sf.guard_extra;
        }
    }
    ws.n[lane] = nr;
    // flat run list in point order
    int pre = nr;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    for (int a = 0; a < nr; ++a) ws.flat[pre - nr + a] = (uint8_t)((lane << 1) | a);
    __syncwarp();
    *more = __any_sync(0xffffffffu, nv > v0 + kRunSlots);
    return __any_sync(0xffffffffu, nr > 0);
}

// ---------------------------------------------------------------------------
// Phase 2: tile-local FP32 poses decide the cell of every point whose FP32
// position lies farther than the guard band from a cell boundary (the band
// bounds the FP32 error, so that cell is the one the FP64 pose gives).
// Ambiguous points are re-binned with the FP64 pose, 32 at a time. FP32 maps
// take the FP32 height; FP64 maps take the FP64 height, computed with the
// same operations as the FP64 pose, so an FP64 map equals the one an
// all-FP64 sweep gives while only the height runs on the FP64 pipe.
// ---------------------------------------------------------------------------
template <bool F64>
using CellOf = typename std::conditional<F64, unsigned long long, uint32_t>::type;

// Cell values. FP32 cells hold the raw bits of a height relative to the
// stock: a cell starts at -0 and only ever takes heights below the stock
// (negative), and negative floats order inversely as signed integers, -0
// (INT_MIN) lowest of all -- so the lowest height is the largest integer
// and a cell is lowered by a signed atomicMax on the bits, with no encoding.
// FP64 cells hold the order-preserving encoding of the height (atomicMin).
constexpr uint32_t kCell32Init = 0x80000000u;  // -0: the stock itself
__device__ __forceinline__ uint32_t cell_key(float zrel) { return __float_as_uint(zrel); }
__device__ __forceinline__ unsigned long long cell_key(double z) {
    return enc64((unsigned long long)__double_as_longlong(z));
}
__device__ __forceinline__ bool lowers(uint32_t e, uint32_t cell) { return (int32_t)e > (int32_t)cell; }
__device__ __forceinline__ bool lowers(unsigned long long e, unsigned long long cell) { return e < cell; }
__device__ __forceinline__ void lower_cell(uint32_t* cell, uint32_t e) { atomicMax((int*)cell, (int)e); }
__device__ __forceinline__ void lower_cell(unsigned long long* cell, unsigned long long e) { atomicMin(cell, e); }

// Key below which a height is below the stock: z < stock exactly when
// cell_key(z) < stock_key(stock) (both zeros take the key of -0, the lowest
// of the two, so that -0 is not below +0). Compares integers on the ALU
// instead of a double on GB300's 1/64-rate FP64 pipe.
__device__ __forceinline__ unsigned long long stock_key(double stock) {
    return cell_key(stock == 0.0 ? -0.0 : stock);
}

// FP64 height of edge point (u, v, w) at phase (cos, sin): the z row of the
// FP64 pose, with wzr = w_z + z_ref formed once per run (as pose64 forms it).
__device__ __forceinline__ double height64(double2 cs, double uz, double vz, double wzr) {
    return __fma_rn(cs.x, uz, __fma_rn(cs.y, vz, wzr));
}

// FP32 height of an FP32 map's point relative to the stock: the FP32 pose's
// z with the operations of the sweep's walks, so a point stores the same
// value whether its cell was decided in FP32 or re-binned in FP64.
__device__ __forceinline__ float height32(const Surface& sf, int m, int idx) {
    const float4* t = sf.tool32 + 4 * (size_t)idx;
    const float uz = t[0].w, vz = t[1].w, zb = sf.zrel_f + t[2].x;
    const float2 c = sf.ph32[m];
    return fmaf(c.x, uz, fmaf(c.y, vz, zb));
}

// Re-bin queued points in FP64 (lanes < count take one entry each). Takes
// the tile by value and returns this lane's (re-binned, atomics, cutting)
// counts, so the caller's counters stay in registers; cutting is counted
// here for FP64 maps only (FP32 maps count it from the FP32 pose). The FP64
// pose decides the cell; the height is the map's own: FP64 for FP64 maps,
// the FP32 pose's for FP32 maps (so an FP32 map does not depend on which
// points were ambiguous, i.e. on the tile shape).
template <bool F64>
__device__ __noinline__ uint4 rebin_flush(const Surface& sf, CellOf<F64>* cells, int tx, int ty, int txc, int tyc,
                                          WarpScratch& ws, int p, int count) {
    const int lane = threadIdx.x & 31;
    uint4 c = make_uint4(0u, 0u, 0u, 0u);
    if (lane < count) {
        const int NE = sf.n_teeth * sf.E;
        const int s = ws.q_s[lane], m = ws.q_m[lane], idx = ws.q_idx[lane];
        const Vec9 v = load_vec9(sf.tool64, NE, idx);
        const int32_t n = s - p * sf.steps_per_pass;
        const Pose64 P = pose64(v, sf.ph64[m], path_x(sf, p, n), path_y(sf, p, n), sf.z_ref);
        c.x = 1u;
        float z32 = 0.f;
        if constexpr (!F64) z32 = height32(sf, m, idx);
        if (F64 ? P.z < sf.stock : z32 < 0.f) {
            const long long ig = bin64(P.x, sf.x0, sf.inv_pitch) - (long long)tx * sf.tile_x;
            const long long kg = bin64(P.y, sf.y0, sf.inv_pitch) - (long long)ty * sf.tile_y;
            if (ig >= 0 && ig < txc && kg >= 0 && kg < tyc) {
                CellOf<F64>* cell = cells + (int)kg * sf.tile_x + (int)ig;
                const auto e = F64 ? (CellOf<F64>)cell_key(P.z) : (CellOf<F64>)cell_key(z32);
                if (lowers(e, *cell)) {
                    lower_cell(cell, e);
                    c.y = 1u;
                }
                c.z = F64 ? 1u : 0u;
            }
        }
    }
    __syncwarp();
    // move the tail down
    const int rest = count > 32 ? count - 32 : 0;
    int s = 0, m = 0, idx = 0;
    if (lane < rest) {
        s = ws.q_s[32 + lane];
        m = ws.q_m[32 + lane];
        idx = ws.q_idx[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        ws.q_s[lane] = s;
        ws.q_m[lane] = m;
        ws.q_idx[lane] = idx;
    }
    __syncwarp();
    return c;
}

template <bool F64>
__device__ __forceinline__ void rebin_flush_count(const Surface& sf, const TileCtx<CellOf<F64>>& tc,
                                                  WarpScratch& ws, int p, int count, Counters& cnt) {
    const uint4 c = rebin_flush<F64>(sf, tc.cells, tc.tx, tc.ty, tc.txc, tc.tyc, ws, p, count);
    cnt.rebinned += c.x;
    cnt.atomics += c.y;
    cnt.cutting += c.z;
}

// Queue this iteration's re-bins (warp-cooperative) and flush full batches.
template <bool F64>
__device__ __forceinline__ void rebin_push(const Surface& sf, const TileCtx<CellOf<F64>>& tc, WarpScratch& ws,
                                           int p, bool want, int32_t s, int32_t m, int idx, int& qn, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, want);
    if (!bal) return;
    const int pos = qn + __popc(bal & ((1u << lane) - 1u));
    if (want) {
        ws.q_s[pos] = s;
        ws.q_m[pos] = m;
        ws.q_idx[pos] = idx;
    }
    qn += __popc(bal);
    __syncwarp();
    if (qn >= 32) {
        rebin_flush_count<F64>(sf, tc, ws, p, qn, cnt);
        qn -= 32;
    }
}

// Ambiguous points of FP32 maps (within the guard band of a cell boundary)
// wait in a per-warp queue and are checked 32 at a time against the cells
// they may belong to: their own and the neighbours across the near
// boundaries, clamped to the tile. Those whose FP32 height -- the value a
// re-binned point stores -- is below one of them go on to FP64 re-binning.
// Cell values only decrease, so a check made later than the point's
// evaluation skips no point that could still lower a cell. (FP64 maps
// re-bin every ambiguous point: their cells hold FP64 heights.)
constexpr int kAmbCap = 64;
struct AmbQueue {
    uint32_t ik[kAmbCap];   // (i + 1) | (k + 1) << 16: tile-local cell of the FP32 pose
    uint32_t mdd[kAmbCap];  // phase index | (dx + 1) << 28 | (dy + 1) << 30: the near boundaries
    uint32_t elo[kAmbCap];  // cell key of the point's FP32 height
    int32_t s[kAmbCap], idx[kAmbCap];
};

// Queue this lane's point if `want` (warp-cooperative; i in [-1, txc] and
// k in [-1, tyc], the cells that can have a neighbour in the tile).
__device__ __forceinline__ void amb_push(AmbQueue& aq, bool want, int i, int k, float rx, float ry, float g,
                                         float z, int32_t s, int32_t m, int idx, int& an) {
    const int lane = threadIdx.x & 31;
    const unsigned bal = __ballot_sync(0xffffffffu, want);
    if (!bal) return;
    if (want) {
        const int pos = an + __popc(bal & ((1u << lane) - 1u));
        const int dx = rx < g - 0.5f ? -1 : (rx > 0.5f - g ? 1 : 0);  // (rx, ry from the cell's centre)
        const int dy = ry < g - 0.5f ? -1 : (ry > 0.5f - g ? 1 : 0);
        aq.ik[pos] = (uint32_t)(i + 1) | ((uint32_t)(k + 1) << 16);
        aq.mdd[pos] = (uint32_t)m | ((uint32_t)(dx + 1) << 28) | ((uint32_t)(dy + 1) << 30);
        aq.elo[pos] = cell_key(z);
        aq.s[pos] = s;
        aq.idx[pos] = idx;
    }
    an += __popc(bal);
    __syncwarp();
}

// Check the first min(count, 32) queued points (one per lane), move the rest
// down, and queue the ones that may lower a cell for FP64 re-binning.
__device__ __forceinline__ void amb_flush(const Surface& sf, const TileCtx<uint32_t>& tc, WarpScratch& ws,
                                          AmbQueue& aq, int p, int count, int& qn, Counters& cnt) {
    const int lane = threadIdx.x & 31;
    bool w = false;
    int32_t s = 0, m = 0, idx = 0;
    if (lane < count) {
        const uint32_t ik = aq.ik[lane], mdd = aq.mdd[lane], elo = aq.elo[lane];
        s = aq.s[lane];
        idx = aq.idx[lane];
        m = (int32_t)(mdd & 0x0FFFFFFFu);
        const int i = (int)(ik & 0xFFFFu) - 1, k = (int)(ik >> 16) - 1;
        const int dx = (int)((mdd >> 28) & 3u) - 1, dy = (int)(mdd >> 30) - 1;
        const int i0 = max(min(i, i + dx), 0), i1 = min(max(i, i + dx), tc.txc - 1);
        const int k0 = max(min(k, k + dy), 0), k1 = min(max(k, k + dy), tc.tyc - 1);
        for (int kk = k0; kk <= k1; ++kk)
            for (int ii = i0; ii <= i1; ++ii) w |= lowers(elo, tc.cells[kk * sf.tile_x + ii]);
    }
    __syncwarp();
    const int rest = count > 32 ? count - 32 : 0;
    uint32_t t_ik = 0, t_mdd = 0, t_elo = 0;
    int32_t t_s = 0, t_idx = 0;
    if (lane < rest) {
        t_ik = aq.ik[32 + lane];
        t_mdd = aq.mdd[32 + lane];
        t_elo = aq.elo[32 + lane];
        t_s = aq.s[32 + lane];
        t_idx = aq.idx[32 + lane];
    }
    __syncwarp();
    if (lane < rest) {
        aq.ik[lane] = t_ik;
        aq.mdd[lane] = t_mdd;
        aq.elo[lane] = t_elo;
        aq.s[lane] = t_s;
        aq.idx[lane] = t_idx;
    }
    __syncwarp();
    rebin_push<false>(sf, tc, ws, p, w, s, m, idx, qn, cnt);
}

// Per-warp scratch in front of the tile cells (precision 0 = FP64, else FP32).
__host__ __device__ constexpr size_t sweep_scratch_bytes(int precision, int threads) {
    return (sizeof(WarpScratch) + (precision == 0 ? 0 : sizeof(AmbQueue))) * (size_t)(threads / 32);
}

// An ambiguous point: FP32 maps queue it for the cell check, FP64 maps for
// re-binning. `an` counts the check queue.
template <bool F64>
__device__ __forceinline__ void push_ambiguous(const Surface& sf, const TileCtx<CellOf<F64>>& tc, WarpScratch& ws,
                                               AmbQueue* aq, int p, bool want, int i, int k, float rx, float ry,
                                               float g, float z, int32_t s, int32_t m, int idx,
                                               int& an, int& qn, Counters& cnt) {
    if constexpr (F64) {
        rebin_push<true>(sf, tc, ws, p, want, s, m, idx, qn, cnt);
    } else {
        amb_push(*aq, want, i, k, rx, ry, g, z, s, m, idx, an);
        if (an >= 32) {
            amb_flush(sf, tc, ws, *aq, p, an, qn, cnt);
            an -= 32;
        }
    }
}

// Drain the queues at the end of a task.
template <bool F64>
__device__ __forceinline__ void drain_queues(const Surface& sf, const TileCtx<CellOf<F64>>& tc, WarpScratch& ws,
                                             AmbQueue* aq, int p, int an, int& qn, Counters& cnt) {
    if constexpr (!F64) {
        while (an > 0) {
            amb_flush(sf, tc, ws, *aq, p, an, qn, cnt);
            an = an > 32 ? an - 32 : 0;
        }
    }
    if (qn > 0) rebin_flush_count<F64>(sf, tc, ws, p, qn, cnt);
    qn = 0;
}

// q = v / len and r = v mod len for 0 <= v < 2^24, from a float reciprocal of
// len with one correction step (the estimate is off by at most one).
__device__ __forceinline__ void divmod_small(int32_t v, int32_t len, float inv_len, int32_t* q, int32_t* r) {
    int32_t d = __float2int_rz((float)v * inv_len);
    d += ((d + 1) * len <= v) ? 1 : 0;
    d -= (d * len > v) ? 1 : 0;
    *q = d;
    *r = v - d * len;
}

// Shared FP32 binning of both walks (tile-local, in cells): the point's
// x offset from the phase table and the x and y rows of its table entry
// (already divided by the pitch, the constant parts less half a cell), the
// pass position from the run's anchor and the steps after the run's first
// item:
//     x = fma(ds, fs, dxA) + fma(cos, ux, fma(sin, vx, wx)),
//     y = dyp + fma(cos, uy, fma(sin, vy, wy)),
// coordinates centred on cells: cell = (rint x, rint y), ambiguous within
// the run's guard band gc of a cell boundary, |x - rint x| > 1/2 - gc.

// Item form of phase 2: the task's runs are taken four at a time, one per
// group of L = 8 lanes; each lane evaluates items hl and hl + L of every 2L
// of its group's run, written as two interleaved, mostly predicated chains
// (the runs average ~70 items, so narrower groups waste fewer slots at run
// ends and share the per-run shuffles among more runs). Counted from phase 0
// of the first occurrence (v = t + first_off; the first occurrence is
// complete up to the window's end whenever there is a second one), item t
// lies in revolution q = v / len at phase offset v mod len, q (S - len) + t
// steps after the run's first item; the lane advances (q, offset) by 2L
// items per iteration without a division.
constexpr int kItemLanes = 8;
#ifndef FSM_ITEM_CHAINS
#define FSM_ITEM_CHAINS 2
#endif
constexpr int kItemChains = FSM_ITEM_CHAINS;  // items per lane and iteration (independent chains)
// kTilt: the surface is fed off the X axis; y then moves by fsy per step
// from the run's own anchor, exactly as x does.
template <bool F64, int U = kItemChains, bool kTilt = false>
__device__ __forceinline__ void sweep_items(const Surface& sf, const TileCtx<CellOf<F64>>& tc, const PassFrame& pf,
                                            int K, int g, int p, WarpScratch& ws, AmbQueue* aq,
                                            const float4 (&t4)[3], float zb_lane, Counters& cnt) {
    using Cell = CellOf<F64>;
    constexpr int L = kItemLanes;
    const int lane = threadIdx.x & 31;
    const int hl = lane & (L - 1), grp = lane / L;
    const int S = sf.S;
    const bool back = pass_reversed(sf, p);
    // cells per step; back on a return pass
    const float fs32 = kTilt ? (back ? -sf.fscx_f : sf.fscx_f) : (back ? -sf.fsc_f : sf.fsc_f);
    const float fsy32 = kTilt ? (back ? -sf.fscy_f : sf.fscy_f) : 0.f;
    const float dyp = pf.dy;
    const float2* __restrict__ ph32 = sf.ph32;
    const double2* __restrict__ ph64 = sf.ph64;
    const int NE = sf.n_teeth * sf.E;
    const double zr = sf.z_ref;
    const unsigned long long below_key = stock_key(sf.stock);
    const int tile_x = sf.tile_x;
    Cell* cells = tc.cells;
    const int txc = tc.txc, tyc = tc.tyc;
    int R = ws.n[lane];
    for (int o = 16; o > 0; o >>= 1) R += __shfl_xor_sync(0xffffffffu, R, o);
    int qn = 0;  // queued re-bins (warp-uniform)
    int an = 0;  // queued ambiguous points (warp-uniform)
    for (int q = 0; q < R; q += 32 / L) {
        const int ri = q + grp;
        const bool has = ri < R;
        const int code = has ? (int)ws.flat[ri] : 0;
        const int o = code >> 1, a = code & 1;
        RunRec r = ws.run[o][a];
        if (!has) {  // a well-formed empty run: its (unused) item indices stay at phase 0
            r.m0 = 0; r.len = 1; r.occ0 = 0; r.first_off = 0; r.len0 = 1; r.k_last = 0; r.len_last = 0;
            r.dxA = 0.f; r.g_cells = 0.f;
        }
        const float ux = __shfl_sync(0xffffffffu, t4[0].x, o), vx = __shfl_sync(0xffffffffu, t4[0].y, o);
        const float wx = __shfl_sync(0xffffffffu, t4[0].z, o), uz = __shfl_sync(0xffffffffu, t4[0].w, o);
        const float uy = __shfl_sync(0xffffffffu, t4[1].x, o), vy = __shfl_sync(0xffffffffu, t4[1].y, o);
        const float wy = __shfl_sync(0xffffffffu, t4[1].z, o), vz = __shfl_sync(0xffffffffu, t4[1].w, o);
        const float zb = __shfl_sync(0xffffffffu, zb_lane, o);
        const int idx = K * sf.E + g * 32 + o;
        double uz64 = 0.0, vz64 = 0.0, wz64 = 0.0;
        if constexpr (F64) {
            uz64 = __ldg(sf.tool64 + 2 * NE + idx);
            vz64 = __ldg(sf.tool64 + 5 * NE + idx);
            wz64 = __dadd_rn(__ldg(sf.tool64 + 8 * NE + idx), zr);  // w_z + z_ref
        }
        const int tot = has ? rec_total(r) : 0;
        int tmax = tot;
        for (int o2 = L; o2 < 32; o2 <<= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o2));
        const int32_t sA = r.occ0 + r.first_off;
        const float gc = r.g_cells;
        float dyA = dyp;  // tilted: the pass's y at the run's first step, in cells
        if constexpr (kTilt) {
            const int32_t n0 = sA - p * sf.steps_per_pass;
            dyA = df_affine(pf.dy, pf.dy_lo, back ? sf.steps_per_pass - 1 - n0 : n0, sf.fscy_hi, sf.fscy_lo);
        }
        // Cells of a point whose FP32 cell is ambiguous lie within M cells of
        // it: M = 1 while the band is under a cell (the host keeps FP32 maps'
        // bands under half a cell); FP64 maps at very fine pitch widen it, and
        // from a band of half a cell every point is ambiguous (FP64 re-binned).
        const float hg = gc >= 0.5f ? -1.0f : 0.5f - gc;
        const int M = F64 ? max(1, (int)ceilf(gc)) : 1;
        const int32_t len = r.len, gap = S - len;
        const float inv_len = 1.0f / (float)len;
        // lane hl takes items hl + k L (k < U) of every U L: item index
        // (revolution q, phase offset o), advanced by L items between its U
        // chains and by U L items per iteration without a division
        int32_t dUL, rUL, dl, rl, q0, o0;
        divmod_small(U * L, len, inv_len, &dUL, &rUL);
        divmod_small(L, len, inv_len, &dl, &rl);
        divmod_small(hl + r.first_off, len, inv_len, &q0, &o0);
        // chain k's next item: its phase index mn (< 2S: the table holds two
        // turns) and its steps after the run's first item dn; both advance by
        // U L items per iteration, the phase wrapping within the run's arc
        int32_t mn[U], dn[U];
        float2 cn[U];  // phase-table entries of the next iteration, loaded one iteration ahead
        {
            int32_t o = o0, q = q0;
#pragma unroll
            for (int k = 0; k < U; ++k) {
                if (k > 0) {
                    o += rl;
                    q += dl;
                    if (o >= len) { o -= len; ++q; }
                }
                mn[k] = r.m0 + o;
                dn[k] = hl + k * L + q * gap;
                cn[k] = __ldg(ph32 + mn[k]);
            }
        }
        const int32_t m_end = r.m0 + len, dn_step = U * L + dUL * gap;
        for (int base = 0; base < tmax; base += U * L) {
            int32_t ds[U], mi[U];
            float2 cs[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                ds[k] = dn[k];
                mi[k] = mn[k];
                cs[k] = cn[k];
                mn[k] += rUL;
                dn[k] += dn_step;
                if (mn[k] >= m_end) { mn[k] -= len; dn[k] += gap; }
                cn[k] = __ldg(ph32 + mn[k]);
            }
            bool push_any = false;
            bool pk[U];
            int ik[U], kk[U];
            float rxk[U], ryk[U], zk[U];
#pragma unroll
            for (int k = 0; k < U; ++k) {
                const bool v = base + hl + k * L < tot;
                const float2 c = cs[k];
                cnt.evaluated += (unsigned)v;
                const float z = fmaf(c.x, uz, fmaf(c.y, vz, zb));
                const float fx = fmaf((float)ds[k], fs32, r.dxA) + fmaf(c.x, ux, fmaf(c.y, vx, wx));
                const float fy = kTilt ? fmaf((float)ds[k], fsy32, dyA) + fmaf(c.x, uy, fmaf(c.y, vy, wy))
                                       : dyp + fmaf(c.x, uy, fmaf(c.y, vy, wy));
                // the cell by one rounding conversion each (coordinates are
                // centred on cells), the offset from its centre by an exact
                // subtraction (Sterbenz)
                const int ix = __float2int_rn(fx), ky = __float2int_rn(fy);
                const float rx = fx - __int2float_rn(ix), ry = fy - __int2float_rn(ky);
                Cell e;
                bool cut;
                if constexpr (F64) {  // below the stock by the FP64 height
                    e = cell_key(height64(__ldg(ph64 + mi[k]), uz64, vz64, wz64));
                    cut = v && e < below_key;
                } else {
                    cut = v && z < 0.f;
                    e = cell_key(z);
                }
                const bool in = cut && (unsigned)ix < (unsigned)txc && (unsigned)ky < (unsigned)tyc;
                // within gc of a cell boundary: |r| > 1/2 - gc on either axis
                const bool amb = fmaxf(fabsf(rx), fabsf(ry)) > hg;
                const bool upd = in && !amb;
                // FP32 maps count the FP32 cell; FP64 maps count ambiguous points when re-binned
                cnt.cutting += F64 ? (unsigned)upd : (unsigned)in;
                const int ci = ky * tile_x + ix;
                const Cell cv = upd ? cells[ci] : (Cell)0;
                if (upd && lowers(e, cv)) {
                    lower_cell(cells + ci, e);
                    ++cnt.atomics;
                }
                pk[k] = cut && amb;  // pushed if near the tile (tested below, rarely reached)
                push_any |= pk[k];
                ik[k] = ix;
                kk[k] = ky;
                rxk[k] = rx;
                ryk[k] = ry;
                zk[k] = z;
            }
            if (__any_sync(0xffffffffu, push_any)) {
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const bool near = ik[k] >= -M && ik[k] <= txc - 1 + M && kk[k] >= -M && kk[k] <= tyc - 1 + M;
                    push_ambiguous<F64>(sf, tc, ws, aq, p, pk[k] && near, ik[k], kk[k], rxk[k], ryk[k], gc, zk[k],
                                        sA + ds[k], mi[k], idx, an, qn, cnt);
                }
            }
        }
    }
    drain_queues<F64>(sf, tc, ws, aq, p, an, qn, cnt);
}

// Phase form of phase 2. The task's runs are taken four at a time, one per
// group of L = 8 lanes, and every lane takes phase offsets of its run.
// Height, y cell and the point's x offset depend on the spindle phase alone,
// so they are computed once per offset; the revolutions of that phase differ
// only by a shift of S fs in x, and those whose x lies within the tile (plus
// M cells and half a cell each side: the ambiguous neighbours, and margin for
// the rounding of the linear revolution model) are found in closed form and
// visited two at a time -- a tile some whole number of revolutions of feed
// wide keeps that number nearly constant across lanes. Each visit bins
// exactly as an item of the item form (same x and y arithmetic, guard band
// and FP64 re-binning), so both forms give the same maps and counts.
template <bool F64>
__device__ __forceinline__ void sweep_phases(const Surface& sf, const TileCtx<CellOf<F64>>& tc, float dyp, int K,
                                             int g, int p, WarpScratch& ws, AmbQueue* aq, const float4 (&t4)[3],
                                             float zb_lane, Counters& cnt) {
    using Cell = CellOf<F64>;
    const int lane = threadIdx.x & 31;
    constexpr int L = kItemLanes;
    const int hl = lane & (L - 1), grp = lane / L;
    const int S = sf.S;
    const float fS = (float)S;
    const bool back = pass_reversed(sf, p);
    const float fs32 = back ? -sf.fsc_f : sf.fsc_f;  // cells per step; back on a return pass
    const float2* __restrict__ ph32 = sf.ph32;
    const double2* __restrict__ ph64 = sf.ph64;
    const int NE = sf.n_teeth * sf.E;
    const double zr = sf.z_ref;
    const unsigned long long below_key = stock_key(sf.stock);
    const int tile_x = sf.tile_x;
    Cell* cells = tc.cells;
    const int txc = tc.txc, tyc = tc.tyc;
    const float inv_rev = 1.0f / (fS * fs32);  // revolutions per cell of x
    int R = ws.n[lane];
    for (int o = 16; o > 0; o >>= 1) R += __shfl_xor_sync(0xffffffffu, R, o);
    int qn = 0;  // queued re-bins (warp-uniform)
    int an = 0;  // queued ambiguous points (warp-uniform)
    for (int q = 0; q < R; q += 32 / L) {
        const int ri = q + grp;
        const bool has = ri < R;
        const int code = has ? (int)ws.flat[ri] : 0;
        const int o = code >> 1, a = code & 1;
        RunRec r = ws.run[o][a];
        if (!has) {  // a well-formed empty run (no offsets; its fields stay in range)
            r.m0 = 0; r.len = 0; r.occ0 = 0; r.first_off = 0; r.len0 = 0; r.k_last = 0; r.len_last = 0;
            r.dxA = 0.f; r.g_cells = 0.f;
        }
        const int len = r.len;
        const float ux = __shfl_sync(0xffffffffu, t4[0].x, o), vx = __shfl_sync(0xffffffffu, t4[0].y, o);
        const float wx = __shfl_sync(0xffffffffu, t4[0].z, o), uz = __shfl_sync(0xffffffffu, t4[0].w, o);
        const float uy = __shfl_sync(0xffffffffu, t4[1].x, o), vy = __shfl_sync(0xffffffffu, t4[1].y, o);
        const float wy = __shfl_sync(0xffffffffu, t4[1].z, o), vz = __shfl_sync(0xffffffffu, t4[1].w, o);
        const float zb = __shfl_sync(0xffffffffu, zb_lane, o);
        const int idx = K * sf.E + g * 32 + o;
        double uz64 = 0.0, vz64 = 0.0, wz64 = 0.0;
        if constexpr (F64) {
            uz64 = __ldg(sf.tool64 + 2 * NE + idx);
            vz64 = __ldg(sf.tool64 + 5 * NE + idx);
            wz64 = __dadd_rn(__ldg(sf.tool64 + 8 * NE + idx), zr);  // w_z + z_ref
        }
        int lmax = len;
        for (int o2 = L; o2 < 32; o2 <<= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o2));
        const int32_t sA = r.occ0 + r.first_off;
        const float gc = r.g_cells;
        // the cells a point may belong to lie within M cells of its FP32 cell
        // (see the item form)
        const float hg = gc >= 0.5f ? -1.0f : 0.5f - gc;
        const int M = F64 ? max(1, (int)ceilf(gc)) : 1;
        // x range of the visits, tile-local cells; k increases toward the
        // far end on a forward pass and toward the near end on a return pass
        const float x_near = -((float)M + 1.0f), x_far = (float)(txc + M);  // (centred coordinates)
        const float xk_lo = back ? x_far : x_near, xk_hi = back ? x_near : x_far;
        const float d_first = (float)(r.occ0 - sA);  // steps from the run's first item to phase 0 of its first turn
        const float klo_c = xk_lo * inv_rev, khi_c = xk_hi * inv_rev;
        const int f0 = r.first_off, f1 = r.first_off + r.len0;
        // the phase-table entry of the next offset is loaded one round ahead
        // (the table does not stay in the L1 left beside a large tile)
        float2 c_next = __ldg(ph32 + r.m0 + (hl < len ? hl : 0));
        for (int ob = 0; ob < lmax; ob += L) {
            const int off = ob + hl;
            const bool vo = off < len;
            const int offc = vo ? off : 0;
            const int32_t m = r.m0 + offc;  // < 2S: the table holds two turns
            const float2 c = c_next;
            c_next = __ldg(ph32 + r.m0 + (off + L < len ? off + L : 0));
            const float z = fmaf(c.x, uz, fmaf(c.y, vz, zb));
            const float px = fmaf(c.x, ux, fmaf(c.y, vx, wx));
            const float fy = dyp + fmaf(c.x, uy, fmaf(c.y, vy, wy));
            const int ky = __float2int_rn(fy);  // the cell: one conversion, its centre's offset by subtraction
            const float ry = fy - __int2float_rn(ky);
            Cell e;
            bool below;
            if constexpr (F64) {  // below the stock by the FP64 height
                e = cell_key(height64(__ldg(ph64 + m), uz64, vz64, wz64));
                below = e < below_key;
            } else {
                below = z < 0.f;
                e = cell_key(z);
            }
            const bool row = vo && below && ky >= -M && ky <= tyc - 1 + M;
            // revolutions of this phase inside the run's step window: the
            // first only for offsets it covers, the last only below its length
            const int kb = (unsigned)(offc - f0) < (unsigned)(f1 - f0) ? 0 : 1;
            const int ke = r.k_last - ((offc >= r.len_last && r.k_last != 0) ? 1 : 0);
            // ... and within the x range: revolution k is d0 + k S steps after
            // the run's first item, at x ~ x0 + k S fs
            const float d0 = d_first + (float)offc;
            const float x0 = fmaf(d0, fs32, r.dxA) + px;
            const int k0 = max(kb, __float2int_ru(fmaf(-x0, inv_rev, klo_c)));
            const int k1 = min(ke, __float2int_rd(fmaf(-x0, inv_rev, khi_c)));
            const int n_it = row ? max(k1 - k0 + 1, 0) : 0;
            const int n_max = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_it);
            const bool ky_in = (unsigned)ky < (unsigned)tyc;
            const float dy = fabsf(ry);
            float ds = fmaf((float)k0, fS, d0);  // steps after the run's first item (an exact integer)
            for (int kk = 0; kk < n_max; kk += 2) {
                const bool va = kk < n_it, vb = kk + 1 < n_it;
                const float dsb = ds + fS;
                const float fxa = fmaf(ds, fs32, r.dxA) + px;
                const float fxb = fmaf(dsb, fs32, r.dxA) + px;
                const int ia = __float2int_rn(fxa), ib = __float2int_rn(fxb);
                const float rxa = fxa - __int2float_rn(ia), rxb = fxb - __int2float_rn(ib);
                cnt.evaluated += (unsigned)va + (unsigned)vb;
                const bool in_a = va && ky_in && (unsigned)ia < (unsigned)txc;
                const bool in_b = vb && ky_in && (unsigned)ib < (unsigned)txc;
                const bool amb_a = fmaxf(fabsf(rxa), dy) > hg;  // within gc of a cell boundary
                const bool amb_b = fmaxf(fabsf(rxb), dy) > hg;
                const bool upd_a = in_a && !amb_a, upd_b = in_b && !amb_b;
                cnt.cutting += F64 ? (unsigned)upd_a + (unsigned)upd_b : (unsigned)in_a + (unsigned)in_b;
                const int cia = ky * tile_x + ia, cib = ky * tile_x + ib;
                const Cell cva = upd_a ? cells[cia] : (Cell)0;
                const Cell cvb = upd_b ? cells[cib] : (Cell)0;
                if (upd_a && lowers(e, cva)) {
                    lower_cell(cells + cia, e);
                    ++cnt.atomics;
                }
                if (upd_b && lowers(e, cvb)) {
                    lower_cell(cells + cib, e);
                    ++cnt.atomics;
                }
                // (va, vb: ky in [-M, tyc - 1 + M], below the stock)
                const bool pa = va && amb_a, pb = vb && amb_b;  // pushed if near the tile (tested below)
                if (__any_sync(0xffffffffu, pa || pb)) {
                    const bool near_a = ia >= -M && ia <= txc - 1 + M, near_b = ib >= -M && ib <= txc - 1 + M;
                    push_ambiguous<F64>(sf, tc, ws, aq, p, pa && near_a, ia, ky, rxa, ry, gc, z, sA + (int32_t)ds, m,
                                        idx, an, qn, cnt);
                    push_ambiguous<F64>(sf, tc, ws, aq, p, pb && near_b, ib, ky, rxb, ry, gc, z,
                                        sA + (int32_t)dsb, m, idx, an, qn, cnt);
                }
                ds = dsb + fS;
            }
        }
    }
    drain_queues<F64>(sf, tc, ws, aq, p, an, qn, cnt);
}

// Position of the n-th set bit (0-based) of x, for n < popc(x): halve the
// word five times, keeping the half that holds it.
__device__ __forceinline__ int nth_set_bit(uint32_t x, int n) {
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t low = (1u << sh) - 1u;
        const int c = __popc(x & low);
        if (n >= c) {
            n -= c;
            x >>= sh;
            pos += sh;
        } else {
            x &= low;
        }
    }
    return pos;
}

// Revolutions k (integers) at which v0 + k rev lies in [lo, hi], for one
// coordinate of a phase offset's visits; the caller intersects the ranges
// of x and y with the run's own revolutions [kb, ke]. A coordinate that
// barely moves between revolutions (|rev| under 1e-4 cells: y on a feed
// near +X, x near +Y) is tested once, widened by its drift over the run.
__device__ __forceinline__ void rev_range(float v0, float rev, float lo, float hi, int kb, int ke, int* k0,
                                          int* k1) {
    if (fabsf(rev) < 1e-4f) {
        const float drift = fabsf(rev) * (float)(ke - kb + 1) + 1.0f;
        const bool in = v0 >= lo - drift && v0 <= hi + drift;
        *k0 = in ? kb : 1;
        *k1 = in ? ke : 0;
        return;
    }
    const float inv = 1.0f / rev;
    const float a = (lo - v0) * inv, b = (hi - v0) * inv;
    *k0 = max(kb, __float2int_ru(fminf(a, b)));
    *k1 = min(ke, __float2int_rd(fmaxf(a, b)));
}

// Phase form of a tilted feed: as sweep_phases, but a revolution moves the
// point along both map axes (S fsx and S fsy cells), so every visit bins y
// as well, and the revolutions visited are those whose x and y both lie
// within the tile widened by M cells and half a cell (closed form per
// coordinate). Each visit bins exactly as the tilted item form (same x and y
// arithmetic, guard band and FP64 re-binning), so both forms give the same
// maps and counts. Unlike the item form's step windows, which come from the
// turned tile's bounding box, the ranges test the tile itself.
template <bool F64>
__device__ __forceinline__ void sweep_phases_tilted(const Surface& sf, const TileCtx<CellOf<F64>>& tc,
                                                    const PassFrame& pf, int K, int g, int p, WarpScratch& ws,
                                                    AmbQueue* aq, const float4 (&t4)[3], float zb_lane,
                                                    Counters& cnt) {
    using Cell = CellOf<F64>;
    const int lane = threadIdx.x & 31;
    constexpr int L = kItemLanes;
    const int hl = lane & (L - 1), grp = lane / L;
    const int S = sf.S;
    const float fS = (float)S;
    const bool back = pass_reversed(sf, p);
    const float fsx = back ? -sf.fscx_f : sf.fscx_f, fsy = back ? -sf.fscy_f : sf.fscy_f;  // cells per step
    const float rev_x = fS * fsx, rev_y = fS * fsy;  // cells per revolution
    const float2* __restrict__ ph32 = sf.ph32;
    const double2* __restrict__ ph64 = sf.ph64;
    const int NE = sf.n_teeth * sf.E;
    const double zr = sf.z_ref;
    const unsigned long long below_key = stock_key(sf.stock);
    const int tile_x = sf.tile_x;
    Cell* cells = tc.cells;
    const int txc = tc.txc, tyc = tc.tyc;
    int R = ws.n[lane];
    for (int o = 16; o > 0; o >>= 1) R += __shfl_xor_sync(0xffffffffu, R, o);
    int qn = 0;  // queued re-bins (warp-uniform)
    int an = 0;  // queued ambiguous points (warp-uniform)
    for (int q = 0; q < R; q += 32 / L) {
        const int ri = q + grp;
        const bool has = ri < R;
        const int code = has ? (int)ws.flat[ri] : 0;
        const int o = code >> 1, a = code & 1;
        RunRec r = ws.run[o][a];
        if (!has) {  // a well-formed empty run (no offsets; its fields stay in range)
            r.m0 = 0; r.len = 0; r.occ0 = 0; r.first_off = 0; r.len0 = 0; r.k_last = 0; r.len_last = 0;
            r.dxA = 0.f; r.g_cells = 0.f;
        }
        const int len = r.len;
        const float ux = __shfl_sync(0xffffffffu, t4[0].x, o), vx = __shfl_sync(0xffffffffu, t4[0].y, o);
        const float wx = __shfl_sync(0xffffffffu, t4[0].z, o), uz = __shfl_sync(0xffffffffu, t4[0].w, o);
        const float uy = __shfl_sync(0xffffffffu, t4[1].x, o), vy = __shfl_sync(0xffffffffu, t4[1].y, o);
        const float wy = __shfl_sync(0xffffffffu, t4[1].z, o), vz = __shfl_sync(0xffffffffu, t4[1].w, o);
        const float zb = __shfl_sync(0xffffffffu, zb_lane, o);
        const int idx = K * sf.E + g * 32 + o;
        double uz64 = 0.0, vz64 = 0.0, wz64 = 0.0;
        if constexpr (F64) {
            uz64 = __ldg(sf.tool64 + 2 * NE + idx);
            vz64 = __ldg(sf.tool64 + 5 * NE + idx);
            wz64 = __dadd_rn(__ldg(sf.tool64 + 8 * NE + idx), zr);  // w_z + z_ref
        }
        int lmax = len;
        for (int o2 = L; o2 < 32; o2 <<= 1) lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o2));
        const int32_t sA = r.occ0 + r.first_off;
        const float gc = r.g_cells;
        const float hg = gc >= 0.5f ? -1.0f : 0.5f - gc;
        const int M = F64 ? max(1, (int)ceilf(gc)) : 1;
        // the pass's y at the run's first step, as in the tilted item form
        const int32_t n0 = sA - p * sf.steps_per_pass;
        const float dyA = df_affine(pf.dy, pf.dy_lo, back ? sf.steps_per_pass - 1 - n0 : n0, sf.fscy_hi, sf.fscy_lo);
        // the tile widened by M cells and half a cell (centred coordinates)
        const float lo_x = -((float)M + 1.0f), hi_x = (float)(txc + M);
        const float lo_y = -((float)M + 1.0f), hi_y = (float)(tyc + M);
        const float d_first = (float)(r.occ0 - sA);  // steps from the run's first item to phase 0 of its first turn
        const int f0 = r.first_off, f1 = r.first_off + r.len0;
        float2 c_next = __ldg(ph32 + r.m0 + (hl < len ? hl : 0));
        for (int ob = 0; ob < lmax; ob += L) {
            const int off = ob + hl;
            const bool vo = off < len;
            const int offc = vo ? off : 0;
            const int32_t m = r.m0 + offc;  // < 2S: the table holds two turns
            const float2 c = c_next;
            c_next = __ldg(ph32 + r.m0 + (off + L < len ? off + L : 0));
            const float z = fmaf(c.x, uz, fmaf(c.y, vz, zb));
            const float px = fmaf(c.x, ux, fmaf(c.y, vx, wx));
            const float py = fmaf(c.x, uy, fmaf(c.y, vy, wy));
            Cell e;
            bool below;
            if constexpr (F64) {  // below the stock by the FP64 height
                e = cell_key(height64(__ldg(ph64 + m), uz64, vz64, wz64));
                below = e < below_key;
            } else {
                below = z < 0.f;
                e = cell_key(z);
            }
            // revolutions of this phase inside the run's step window ...
            const int kb = (offc >= f0 && offc < f1) ? 0 : 1;
            const int ke = r.k_last == 0 ? 0 : (offc < r.len_last ? r.k_last : r.k_last - 1);
            // ... and over the tile along both axes: revolution k is d0 + k S
            // steps after the run's first item, at (x0, y0) + k S (fsx, fsy)
            const float d0 = d_first + (float)offc;
            const float x0 = fmaf(d0, fsx, r.dxA) + px;
            const float y0 = fmaf(d0, fsy, dyA) + py;
            int kx0, kx1, ky0, ky1;
            rev_range(x0, rev_x, lo_x, hi_x, kb, ke, &kx0, &kx1);
            rev_range(y0, rev_y, lo_y, hi_y, kb, ke, &ky0, &ky1);
            const int k0 = max(kx0, ky0), k1 = min(kx1, ky1);
            const int n_it = (vo && below) ? max(k1 - k0 + 1, 0) : 0;
            const int n_max = (int)__reduce_max_sync(0xffffffffu, (unsigned)n_it);
            float ds = fmaf((float)k0, fS, d0);  // steps after the run's first item (an exact integer)
            for (int kk = 0; kk < n_max; kk += 2) {
                const bool va = kk < n_it, vb = kk + 1 < n_it;
                const float dsb = ds + fS;
                const float fxa = fmaf(ds, fsx, r.dxA) + px, fya = fmaf(ds, fsy, dyA) + py;
                const float fxb = fmaf(dsb, fsx, r.dxA) + px, fyb = fmaf(dsb, fsy, dyA) + py;
                const int ia = __float2int_rn(fxa), ja = __float2int_rn(fya);
                const int ib = __float2int_rn(fxb), jb = __float2int_rn(fyb);
                const float rxa = fxa - __int2float_rn(ia), rya = fya - __int2float_rn(ja);
                const float rxb = fxb - __int2float_rn(ib), ryb = fyb - __int2float_rn(jb);
                cnt.evaluated += (unsigned)va + (unsigned)vb;
                const bool in_a = va && (unsigned)ia < (unsigned)txc && (unsigned)ja < (unsigned)tyc;
                const bool in_b = vb && (unsigned)ib < (unsigned)txc && (unsigned)jb < (unsigned)tyc;
                const bool amb_a = fmaxf(fabsf(rxa), fabsf(rya)) > hg;  // within gc of a cell boundary
                const bool amb_b = fmaxf(fabsf(rxb), fabsf(ryb)) > hg;
                const bool upd_a = in_a && !amb_a, upd_b = in_b && !amb_b;
                cnt.cutting += F64 ? (unsigned)upd_a + (unsigned)upd_b : (unsigned)in_a + (unsigned)in_b;
                const int cia = ja * tile_x + ia, cib = jb * tile_x + ib;
                const Cell cva = upd_a ? cells[cia] : (Cell)0;
                const Cell cvb = upd_b ? cells[cib] : (Cell)0;
                if (upd_a && lowers(e, cva)) {
                    lower_cell(cells + cia, e);
                    ++cnt.atomics;
                }
                if (upd_b && lowers(e, cvb)) {
                    lower_cell(cells + cib, e);
                    ++cnt.atomics;
                }
                const bool pa = va && amb_a, pb = vb && amb_b;  // pushed if near the tile (tested below)
                if (__any_sync(0xffffffffu, pa || pb)) {
                    const bool near_a = ia >= -M && ia <= txc - 1 + M && ja >= -M && ja <= tyc - 1 + M;
                    const bool near_b = ib >= -M && ib <= txc - 1 + M && jb >= -M && jb <= tyc - 1 + M;
                    push_ambiguous<F64>(sf, tc, ws, aq, p, pa && near_a, ia, ja, rxa, rya, gc, z, sA + (int32_t)ds, m,
                                        idx, an, qn, cnt);
                    push_ambiguous<F64>(sf, tc, ws, aq, p, pb && near_b, ib, jb, rxb, ryb, gc, z,
                                        sA + (int32_t)dsb, m, idx, an, qn, cnt);
                }
                ds = dsb + fS;
            }
        }
    }
    drain_queues<F64>(sf, tc, ws, aq, p, an, qn, cnt);
}

__device__ __forceinline__ int find_surface(const int* tile_base, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tile_base[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Persistent tile sweep. Tiles of all surfaces form one index space
// (tile_base[s] = first tile of surface s); CTAs take tiles in a static
// stride, or from *queue when it is not NULL. Inside a tile, warps take
// (pass, tooth, 32-point group) tasks from a shared counter.
// kTilt: the launch may hold surfaces fed off the X axis (y stepping along
// the feed in either form; these instantiations are phase-capable); the
// others run as in the plain phase-capable instantiation.
template <bool FP64, bool kCount, bool kPhases, bool kTilt = false>
__global__ void __launch_bounds__(512, 1) sweep_kernel(const Surface* __restrict__ surfs, int n_surf,
                                                       const int* __restrict__ tile_base, int total_tiles,
                                                       int* queue, long long* counters) {
    using Cell = typename std::conditional<FP64, unsigned long long, uint32_t>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_task, s_tile;
    __shared__ TileShared ts;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    // [WarpScratch x warps][AmbQueue x warps, FP32 only][tile cells]
    WarpScratch* wscr = reinterpret_cast<WarpScratch*>(smem);
    AmbQueue* aqs = reinterpret_cast<AmbQueue*>(smem + sizeof(WarpScratch) * nwarps);
    Cell* cells = reinterpret_cast<Cell*>(smem + sweep_scratch_bytes(FP64 ? 0 : 1, nwarps * 32));
    WarpScratch& ws = wscr[warp];
    Counters cnt = {0, 0, 0, 0};

    int iter = 0;
    while (true) {
        if (threadIdx.x == 0) {
            s_tile = queue ? atomicAdd(queue, 1) : (int)blockIdx.x + iter * (int)gridDim.x;
            s_task = 0;
        }
        ++iter;
        __syncthreads();
        const int t = s_tile;
        if (t >= total_tiles) break;
        const int sidx = (n_surf == 1 || tile_base == nullptr) ? 0 : find_surface(tile_base, n_surf, t);
        const Surface& sf = surfs[sidx];
        const int lt = t - (tile_base ? tile_base[sidx] : 0);
        TileCtx<Cell> tc;
        tc.cells = cells;
        tc.tx = lt % sf.ntx;
        tc.ty = lt / sf.ntx;
        tc.txc = min(sf.tile_x, sf.nx - tc.tx * sf.tile_x);
        tc.tyc = min(sf.tile_y, sf.ny - tc.ty * sf.tile_y);
        tc.X0 = sf.x0 + (double)(tc.tx * sf.tile_x) * sf.pitch;
        tc.Y0 = sf.y0 + (double)(tc.ty * sf.tile_y) * sf.pitch;
        const int ncell = sf.tile_x * sf.tile_y;
        Cell init;
        if constexpr (FP64) init = (Cell)enc64((unsigned long long)__double_as_longlong(sf.stock));
        else init = (Cell)kCell32Init;  // FP32 cells hold heights relative to the stock
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) cells[c] = init;
        fill_tile_shared<kTilt>(sf, tc, ts);
        __syncthreads();
        // Task order: the passes whose line runs nearest the tile's centre
        // (|centre of the y band|, relative to the pass line) first -- their
        // tasks carry the most runs, so the warps' last tasks are short ones
        // and the wait at the end of the tile shrinks. Passes beyond the
        // cached ones keep their index order.
        const int n_cached = min(sf.n_passes, kPassCache);
        if (threadIdx.x < n_cached) {
            const int q = threadIdx.x;
            const float dq = fabsf(ts.ylo[q] + ts.yhi[q]);
            int rank = 0;
            for (int o = 0; o < n_cached; ++o) {
                const float d = fabsf(ts.ylo[o] + ts.yhi[o]);
                rank += (d < dq || (d == dq && o < q)) ? 1 : 0;
            }
            ts.order[rank] = (uint8_t)q;
        }
        __syncthreads();

        const int G = (sf.E + 31) / 32;
        const int n_tasks = sf.n_passes * sf.n_teeth * G;
        // group reject of the tile's first tasks, a warp per 32 tasks: the
        // bounds loads of many tasks are in flight at once, and a warp then
        // skips rejected tasks with one shared load instead of a global one
        const int n_bits = min(n_tasks, kTaskBits);
        for (int w0 = warp * 32; w0 < n_bits; w0 += nwarps * 32) {
            const int t = w0 + lane;
            bool ok = false;
            if (t < n_bits) {
                const int pi = t / (sf.n_teeth * G);
                const int rem = t - pi * sf.n_teeth * G;
                const int p = pi < kPassCache ? (int)ts.order[pi] : pi;
                PassFrame pf;
                pass_band<kTilt>(sf, tc, ts, p, pf);
                const float4 gb = sf.groups[rem];  // rem = K * G + g
                ok = !(gb.y < pf.ylo || gb.x > pf.yhi || gb.z >= ts.zhi);
            }
            const unsigned bits = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) ts.accept[w0 >> 5] = bits;
        }
        __syncthreads();
        // prefix counts of the accept words (warp 0; at most 128 words, four
        // per lane): the accepted tasks are handed out by rank, so no warp
        // takes a rejected one
        const int n_words = (n_bits + 31) >> 5;
        if (warp == 0) {
            int c[4], sum = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int w = lane * 4 + k;
                c[k] = w < n_words ? __popc(ts.accept[w]) : 0;
                sum += c[k];
            }
            int incl = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            int run = incl - sum;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int w = lane * 4 + k;
                if (w < n_words) ts.acc_pre[w] = (uint16_t)run;
                run += c[k];
            }
            if (lane == 31) ts.acc_pre[n_words] = (uint16_t)incl;
        }
        __syncthreads();
        const int n_acc = ts.acc_pre[n_words];
        const float inv_ng = 1.0f / (float)(sf.n_teeth * G), inv_g = 1.0f / (float)G;
        const double tile_x1 = tc.X0 + (double)tc.txc * sf.pitch;
        const double pass_x1 = sf.pass_x0 + (double)(sf.steps_per_pass - 1) * sf.fs;
        bool x_miss = (pass_x1 + sf.reach_x < tc.X0 - 1e-3) || (sf.pass_x0 - sf.reach_x > tile_x1 + 1e-3);
        if (kTilt && sf.tilted) {  // along the feed: the tile's extent against the passes' reach
            const double len = (double)(sf.steps_per_pass - 1) * sf.fs;
            x_miss = ((double)ts.xlo > len + sf.reach_x + 1e-3) || ((double)ts.xhi < -sf.reach_x - 1e-3);
        }
        while (!x_miss) {
            int r = 0;
            if (lane == 0) r = atomicAdd(&s_task, 1);
            r = __shfl_sync(0xffffffffu, r, 0);
            int task;
            if (r < n_acc) {  // the r-th accepted task: its word, then its bit
                bool hit = false;
                int wl = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int w = lane * 4 + k;
                    if (w < n_words && (int)ts.acc_pre[w] <= r && r < (int)ts.acc_pre[w + 1]) {
                        hit = true;
                        wl = w;
                    }
                }
                const unsigned who = __ballot_sync(0xffffffffu, hit);
                if (who == 0u) break;  // (not reached: the prefix counts cover every rank below n_acc)
                const int w = __shfl_sync(0xffffffffu, wl, __ffs(who) - 1);
                task = w * 32 + nth_set_bit(ts.accept[w], r - (int)ts.acc_pre[w]);
            } else {  // tasks beyond the tabulated ones, tested as they are taken
                task = n_bits + (r - n_acc);
                if (task >= n_tasks) break;
            }
            int pi, rem, K, g;  // task = (pi N + K) G + g; float-reciprocal divisions (exact below 2^24)
            if (task < (1 << 24)) {
                divmod_small(task, sf.n_teeth * G, inv_ng, &pi, &rem);
            } else {
                pi = task / (sf.n_teeth * G);
                rem = task - pi * sf.n_teeth * G;
            }
            divmod_small(rem, G, inv_g, &K, &g);  // rem < N G <= 2^21
            const int p = pi < kPassCache ? (int)ts.order[pi] : pi;
            PassFrame pf;
            pass_band<kTilt>(sf, tc, ts, p, pf);
            if (task >= kTaskBits) {
                const float4 gb = sf.groups[K * G + g];
                if (gb.y < pf.ylo || gb.x > pf.yhi || gb.z >= ts.zhi) continue;  // warp-uniform
            }
            AmbQueue* aq = FP64 ? nullptr : aqs + warp;
            bool by_phase = false;
            for (int round = 0;; ++round) {  // (a second round is rare: points with more than kRunSlots runs)
                float4 t4[3];
                float zb;
                bool more = false;
                int items = 0, phases = 0;
                const bool any = warp_runs<kTilt>(sf, ts, pf, K, g, p, ws, t4, zb, round, &more, &items, &phases);
                if (any) {
                    if (round == 0) {
                        // runs that come back for many revolutions share their
                        // per-phase work (phase form); others are walked item by item
                        if constexpr (kPhases) {
                            if (sf.form == FSM_FORM_PHASE) {
                                by_phase = true;
                            } else if (sf.form != FSM_FORM_ITEM) {
                                for (int o = 16; o > 0; o >>= 1) {
                                    items += __shfl_xor_sync(0xffffffffu, items, o);
                                    phases += __shfl_xor_sync(0xffffffffu, phases, o);
                                }
                                // (FP32 tasks of a tilted feed stay item by item: its phase
                                // form evaluates a third fewer poses but costs more per
                                // visit, 30 degrees 2.97 -> 3.42 ms; FP64 gains, 10.5 -> 8.9)
                                by_phase = (FP64 || !(kTilt && sf.tilted)) && phase_form_task<FP64>(items, phases);
                            }
                        }
                        if (sf.form_tasks && lane == 0) atomicAdd(sf.form_tasks + (by_phase ? 1 : 0), 1ull);
                    }
                    bool tilted_phases = false;
                    if constexpr (kTilt) tilted_phases = by_phase && sf.tilted;
                    if (tilted_phases) {
                        if constexpr (kTilt) sweep_phases_tilted<FP64>(sf, tc, pf, K, g, p, ws, aq, t4, zb, cnt);
                    } else if (by_phase)
                        sweep_phases<FP64>(sf, tc, pf.dy, K, g, p, ws, aq, t4, zb, cnt);
                    else if (kTilt && sf.tilted)
                        sweep_items<FP64, kItemChains, kTilt>(sf, tc, pf, K, g, p, ws, aq, t4, zb, cnt);
                    else
                        sweep_items<FP64>(sf, tc, pf, K, g, p, ws, aq, t4, zb, cnt);
                    __syncwarp();
                }
                if (!more) break;
            }
        }
        __syncthreads();

        // decode and store the tile
        if constexpr (FP64) {
            double* out = reinterpret_cast<double*>(sf.heights);
            for (int c = threadIdx.x; c < tc.txc * tc.tyc; c += blockDim.x) {
                const int k = c / tc.txc, i = c - k * tc.txc;
                const unsigned long long e = cells[k * sf.tile_x + i];
                out[(size_t)(tc.ty * sf.tile_y + k) * sf.nx + tc.tx * sf.tile_x + i] =
                    __longlong_as_double((long long)dec64(e));
            }
        } else {
            float* out = reinterpret_cast<float*>(sf.heights);
            const float st = (float)sf.stock;
            const bool vec = ((sf.nx & 3) == 0) && ((tc.txc & 3) == 0) && ((sf.tile_x & 3) == 0) &&
                             ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
            if (vec) {
                const int q = tc.txc >> 2;
                for (int c = threadIdx.x; c < q * tc.tyc; c += blockDim.x) {
                    const int k = c / q, i4 = (c - k * q) << 2;
                    const uint4 e = *reinterpret_cast<const uint4*>(cells + k * sf.tile_x + i4);
                    float4 v;
                    v.x = st + __uint_as_float(e.x);
                    v.y = st + __uint_as_float(e.y);
                    v.z = st + __uint_as_float(e.z);
                    v.w = st + __uint_as_float(e.w);
                    *reinterpret_cast<float4*>(
                        out + (size_t)(tc.ty * sf.tile_y + k) * sf.nx + tc.tx * sf.tile_x + i4) = v;
                }
            } else {
                for (int c = threadIdx.x; c < tc.txc * tc.tyc; c += blockDim.x) {
                    const int k = c / tc.txc, i = c - k * tc.txc;
                    out[(size_t)(tc.ty * sf.tile_y + k) * sf.nx + tc.tx * sf.tile_x + i] =
                        st + __uint_as_float(cells[k * sf.tile_x + i]);
                }
            }
        }
        __syncthreads();
    }
    if constexpr (kCount) warp_flush(cnt, counters);
}

// ===========================================================================
// Roughness: FP64 moments with a fixed reduction tree. Maps are cut into
// chunks of kChunk cells; block b reduces chunk b of the job that owns it
// (chunk_base[j] = first chunk of job j), so one launch serves one map or a
// batch of maps of any sizes. Every sum is taken in the same order whatever
// the launch timing, so results are reproducible bit for bit.
// ===========================================================================
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum (kind 0), min (1) or max (2) of v over the block, in a fixed order;
// every thread gets the result.
template <int KIND>
__device__ __forceinline__ double block_reduce(double v, double* sh /*[32]*/) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    v = KIND == 0 ? warp_sum(v) : KIND == 1 ? warp_min(v) : warp_max(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double x = lane < nw ? sh[lane] : (KIND == 0 ? 0.0 : KIND == 1 ? 1e300 : -1e300);
    x = KIND == 0 ? warp_sum(x) : KIND == 1 ? warp_min(x) : warp_max(x);
    return x;
}

// Min (kind 1) or max (2) of a float over the block (exact); every thread
// gets the result.
template <int KIND>
__device__ __forceinline__ float block_minmax_f(float v, double* sh /*[32]*/) {
    float* sf = reinterpret_cast<float*>(sh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, v, o);
        v = KIND == 1 ? fminf(v, w) : fmaxf(v, w);
    }
    __syncthreads();
    if (lane == 0) sf[warp] = v;
    __syncthreads();
    float x = lane < nw ? sf[lane] : (KIND == 1 ? 3.0e38f : -3.0e38f);
    for (int o = 16; o > 0; o >>= 1) {
        const float w = __shfl_xor_sync(0xffffffffu, x, o);
        x = KIND == 1 ? fminf(x, w) : fmaxf(x, w);
    }
    return x;
}

// Double-float sums for FP32 maps, on the FP32 pipes (GB300 runs FP64 at
// 1/64 of the FP32 rate): unevaluated pairs (hi, lo) added with Knuth's
// two-sum on the high parts (exact and symmetric in its operands, so every
// lane of a butterfly ends with the same pair).
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    float t, e;
    two_sum(a.x, b.x, &t, &e);
    e += a.y + b.y;
    const float hi = t + e;
    return make_float2(hi, e - (hi - t));
}

// Block sum of double-float values in a fixed tree; every thread gets it.
__device__ __forceinline__ double block_sum_df(float2 v, double* sh /*[32]*/) {
    float2* s2 = reinterpret_cast<float2*>(sh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    __syncthreads();
    if (lane == 0) s2[warp] = v;
    __syncthreads();
    float2 x = lane < nw ? s2[lane] : make_float2(0.f, 0.f);
    for (int o = 16; o > 0; o >>= 1)
        x = df_add(x, make_float2(__shfl_xor_sync(0xffffffffu, x.x, o), __shfl_xor_sync(0xffffffffu, x.y, o)));
    return (double)x.x + (double)x.y;
}

// Four block sums of double-float values in one fixed tree (one pair of
// barriers instead of four); thread 0 gets the results. sh: 128 doubles.
__device__ __forceinline__ void block_sum_df4(const float2 (&v)[4], double* sh, double (&out)[4]) {
    float2* s2 = reinterpret_cast<float2*>(sh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    float2 a[4] = {v[0], v[1], v[2], v[3]};
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            a[k] = df_add(a[k], make_float2(__shfl_xor_sync(0xffffffffu, a[k].x, o),
                                            __shfl_xor_sync(0xffffffffu, a[k].y, o)));
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) s2[4 * warp + k] = a[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = lane < nw ? s2[4 * lane + k] : make_float2(0.f, 0.f);
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                a[k] = df_add(a[k], make_float2(__shfl_xor_sync(0xffffffffu, a[k].x, o),
                                                __shfl_xor_sync(0xffffffffu, a[k].y, o)));
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = (double)a[k].x + (double)a[k].y;
    }
}

// FP64 maps' moments on the FP32 pipes (GB300 runs FP64 at 1/64 of the
// FP32 rate): a double as an unevaluated float pair hi + lo, from its bits
// (hi: the top 24 significant bits, truncated; lo: the other 29, rounded to
// a float), |z - (hi + lo)| <= 2^-47 |z|, no FP64 instruction; magnitudes
// outside [2^-60, 2^100] (zero included) take FP64 conversions.
// The rare magnitudes by FP64 conversions, in a call of its own so the
// compiler cannot turn the branch into predicated FP64 instructions that
// every cell would issue.
__device__ __noinline__ float2 split_double_slow(double z) {
    const float hi = (float)z;
    return make_float2(hi, (float)(z - (double)hi));
}

__device__ __forceinline__ float2 split_double(double z) {
    const unsigned hw = (unsigned)__double2hiint(z), lw = (unsigned)__double2loint(z);
    const int e = (int)((hw >> 20) & 0x7FFu) - 1023;
    if (e < -60 || e > 100) return split_double_slow(z);
    const unsigned sign = hw & 0x80000000u;
    // fraction bits 51..29 (hw's 20, lw's top 3) and 28..0 (lw's rest)
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    const unsigned rem = lw & 0x1FFFFFFFu;  // worth rem * 2^(e - 52)
    float lo = 0.f;
    if (rem) lo = __uint_as_float((__float_as_uint(__uint2float_rn(rem)) + ((unsigned)(e - 52) << 23)) | sign);
    return make_float2(hi, lo);
}

// x * y of double-float pairs (the leading product's rounding error by fma).
__device__ __forceinline__ float2 df_mul(float2 x, float2 y) {
    const float p = x.x * y.x;
    const float pe = fmaf(x.x, y.x, -p) + fmaf(x.x, y.y, x.y * y.x);
    const float hi = p + pe;
    return make_float2(hi, pe - (hi - p));
}

__device__ __forceinline__ int find_job(const int* base, int n, int b) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ void chunk_range(const RoughJob& jb, int c, size_t* lo, size_t* hi) {
    *lo = (size_t)c * kChunk;
    const size_t e = *lo + kChunk;
    *hi = e < jb.n ? e : jb.n;
}

// Pass 1: per chunk sum, min, max -> part[b*3 + {0,1,2}]
// Sync words of a set of roughness jobs: pass-1 and pass-2 completion
// counters and the job means (zeroed before pass 1).
struct RoughSync {
    int* done1;
    int* done2;
    double* mean;
};

__device__ __forceinline__ RoughSync rough_sync(void* base, int n_jobs) {
    RoughSync r;
    r.done1 = (int*)base;
    r.done2 = r.done1 + n_jobs;
    r.mean = (double*)((char*)base + ((8 * (size_t)n_jobs + 7) & ~(size_t)7));
    return r;
}

// Called by the whole block: true in the block that completes job j's last
// chunk of this pass (its writes and every other block's are then visible).
__device__ __forceinline__ bool last_chunk_block(int* done, int j, int n_chunks) {
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done + j, 1) == n_chunks - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Chunk sums of FP32 maps are taken about a reference height (the map's
// first cell), so their FP32 leaves carry deviations only; FP64 maps use 0.
__device__ double job_mean(const double* part, int c0, int c1, size_t n, double ref, double* sh) {
    double s = 0.0;
    for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) s += __ldcg(part + 3 * (size_t)c);
    s = block_reduce<0>(s, sh);
    return ref + s / (double)n;
}

// End of pass 1: the block completing job j's last chunk stores its mean.
__device__ __forceinline__ void job_mean_if_last(const RoughJob* __restrict__ jobs,
                                                 const int* __restrict__ chunk_base, const double* part, int n_jobs,
                                                 int j, void* sync, double ref, double* sh) {
    const RoughSync rs = rough_sync(sync, n_jobs);
    const int c0 = chunk_base[j], c1 = chunk_base[j + 1];
    if (last_chunk_block(rs.done1, j, c1 - c0)) {
        const double mu = job_mean(part, c0, c1, jobs[j].n, ref, sh);
        if (threadIdx.x == 0) rs.mean[j] = mu;
    }
}

template <typename T>
__device__ void profile_seg1(const RoughJob* __restrict__ jobs, int item, int per_job, double* ppart, double* sh);
__device__ void finalize_job(const RoughJob* __restrict__ jobs, const int* __restrict__ chunk_base,
                             const double* part, const double* part2, int j, double mu, int per_job,
                             const double* ppart, double* sh);
__device__ void finalize_profiles(const RoughJob& jb, int j, int per_job, const double* ppart);

template <typename T>
__device__ __forceinline__ void rough1_item(const RoughJob* __restrict__ jobs, int n_jobs,
                                            const int* __restrict__ chunk_base, double* part, int total_chunks,
                                            int per_job, void* sync, int b, double* sh) {
    if (b >= total_chunks) {  // items past the chunks are profile segments
        profile_seg1<T>(jobs, b - total_chunks, per_job, part + 7 * (size_t)total_chunks, sh);
        return;
    }
    const int j = find_job(chunk_base, n_jobs, b);
    const RoughJob jb = jobs[j];
    size_t lo, hi;
    chunk_range<T>(jb, b - chunk_base[j], &lo, &hi);
    const T* h = reinterpret_cast<const T*>(jb.h);
    // min and max on the order-preserving keys (exact, on the integer ALU);
    // the sum of z - ref (ref: the map's first cell), each difference one
    // FP64 subtraction split into a float pair, summed in double-float on the
    // FP32 pipes (the split's 2^-47 is then relative to the difference, not
    // to z: maps far from zero keep their texture's precision)
    const double ref = (double)h[0];
    float2 s = make_float2(0.f, 0.f);
    // keys as (high, low) 32-bit words, compared lexicographically
    unsigned mn_h = ~0u, mn_l = ~0u, mx_h = 0u, mx_l = 0u;
#pragma unroll 4
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double z = (double)h[i];
        s = df_add(s, split_double(z - ref));
        const unsigned zh = (unsigned)__double2hiint(z), zl = (unsigned)__double2loint(z);
        const bool neg = (zh >> 31) != 0u;
        const unsigned kh = neg ? ~zh : (zh | 0x80000000u), kl = neg ? ~zl : zl;
        if (kh < mn_h || (kh == mn_h && kl < mn_l)) { mn_h = kh; mn_l = kl; }
        if (kh > mx_h || (kh == mx_h && kl > mx_l)) { mx_h = kh; mx_l = kl; }
    }
    const unsigned long long kmn = ((unsigned long long)mn_h << 32) | mn_l;
    const unsigned long long kmx = ((unsigned long long)mx_h << 32) | mx_l;
    const double sum = block_sum_df(s, sh);
    double mn = kmn == ~0ull ? 1e300 : __longlong_as_double((long long)dec64(kmn));
    double mx = kmx == 0ull ? -1e300 : __longlong_as_double((long long)dec64(kmx));
    mn = block_reduce<1>(mn, sh);
    mx = block_reduce<2>(mx, sh);
    if (threadIdx.x == 0) {
        part[3 * (size_t)b] = sum;
        part[3 * (size_t)b + 1] = mn;
        part[3 * (size_t)b + 2] = mx;
    }
    job_mean_if_last(jobs, chunk_base, part, n_jobs, j, sync, ref, sh);
}

// Mean of job j from its chunk sums, in chunk order (identical in every block).

// Final: the whole block combines job j's chunks (in chunk order) and writes
// the areal values. Chunk partials written by other blocks of the running
// launch are read past L1.
__device__ void finalize_job(const RoughJob* __restrict__ jobs, const int* __restrict__ chunk_base,
                             const double* part, const double* part2, int j, double mu, int per_job,
                             const double* ppart, double* sh) {
    const RoughJob jb = jobs[j];
    const int c0 = chunk_base[j], c1 = chunk_base[j + 1];
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    double mn = 1e300, mx = -1e300;
    for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
        for (int a = 0; a < 4; ++a) v[a] += __ldcg(part2 + 4 * (size_t)c + a);
        mn = fmin(mn, __ldcg(part + 3 * (size_t)c + 1));
        mx = fmax(mx, __ldcg(part + 3 * (size_t)c + 2));
    }
    for (int a = 0; a < 4; ++a) v[a] = block_reduce<0>(v[a], sh);
    mn = block_reduce<1>(mn, sh);
    mx = block_reduce<2>(mx, sh);
    if (threadIdx.x == 0) {
        fsm_roughness_out* out = jb.out;
        const double dn = (double)jb.n;
        out->n = dn;
        out->mean = mu;
        out->zmin = mn;
        out->zmax = mx;
        out->Sa = v[0] / dn;
        out->Sq = sqrt(v[1] / dn);
        out->Sp = mx - mu;
        out->Sv = mu - mn;
        out->Sz = out->Sp + out->Sv;
        if (out->Sq > 0.0) {
            const double sq = out->Sq;
            out->Ssk = (v[2] / dn) / (sq * sq * sq);
            out->Sku = (v[3] / dn) / (sq * sq * sq * sq);
        } else {
            out->Ssk = __longlong_as_double(0x7ff8000000000000ll);
            out->Sku = __longlong_as_double(0x7ff8000000000000ll);
        }
        out->n_rows = jb.n_rows;
        out->n_cols = jb.n_cols;
    }
    finalize_profiles(jb, j, per_job, ppart);
}

// Profiles, cut into the 5 segments of Rz ([floor(s L/5), floor((s+1) L/5))),
// one block per segment in each pass: pass 1 takes each segment's sum, min
// and max, pass 2 its sum of |z - profile mean| (the mean from the five sums,
// in segment order, identical in every block). Item i of a pass is segment
// i mod 5 of profile (i / 5) mod per_job (rows first, then columns) of job
// i / (5 per_job). Partials: ppart[((j per_job + q) 5 + seg) 4 + {sum, min,
// max, |dev|}].
constexpr int kRzSegments = 5;
// Resident blocks per SM the roughness passes are compiled for (registers
// capped so a 25 Mcell map's chunks and profile segments fit in one wave).
constexpr int kRoughBlocksPerSm = 6;

struct ProfileSeg {
    bool valid, row;
    int r, fixed, L, lo, hi;  // profile r of its kind at row/column `fixed`, length L, segment [lo, hi)
    size_t base, stride;      // cell a of the profile: base + a stride
};

__device__ __forceinline__ ProfileSeg profile_seg(const RoughJob& jb, int q, int seg) {
    ProfileSeg ps;
    ps.valid = q < jb.n_rows + jb.n_cols;
    ps.row = q < jb.n_rows;
    ps.r = ps.row ? q : q - jb.n_rows;
    if (ps.row) {
        ps.fixed = jb.n_rows > 0 ? (int)(((long long)(2 * ps.r + 1) * jb.ny) / (2 * jb.n_rows)) : 0;
        ps.base = (size_t)ps.fixed * jb.nx;
        ps.stride = 1;
        ps.L = jb.nx;
    } else {
        ps.fixed = jb.n_cols > 0 ? (int)(((long long)(2 * ps.r + 1) * jb.nx) / (2 * jb.n_cols)) : 0;
        ps.base = (size_t)ps.fixed;
        ps.stride = (size_t)jb.nx;
        ps.L = jb.ny;
    }
    ps.lo = (int)(((long long)seg * ps.L) / kRzSegments);
    ps.hi = (int)(((long long)(seg + 1) * ps.L) / kRzSegments);
    return ps;
}

// Pass 1 of a profile segment: sum (double-float for FP32 maps, each value
// exact), min and max (exact in the map's precision).
template <typename T>
__device__ void profile_seg1(const RoughJob* __restrict__ jobs, int item, int per_job, double* ppart, double* sh) {
    const int j = item / (per_job * kRzSegments), rem = item - j * per_job * kRzSegments;
    const int q = rem / kRzSegments, seg = rem - q * kRzSegments;
    const RoughJob jb = jobs[j];
    const ProfileSeg ps = profile_seg(jb, q, seg);
    if (!ps.valid) return;
    const T* h = reinterpret_cast<const T*>(jb.h);
    double sum, mn, mx;
    if constexpr (sizeof(T) == 4) {
        float2 acc = make_float2(0.f, 0.f);
        float fn = 3.0e38f, fx = -3.0e38f;
        for (int a = ps.lo + threadIdx.x; a < ps.hi; a += blockDim.x) {
            const float z = (float)h[ps.base + (size_t)a * ps.stride];
            acc = df_add(acc, make_float2(z, 0.f));
            fn = fminf(fn, z);
            fx = fmaxf(fx, z);
        }
        sum = block_sum_df(acc, sh);
        mn = (double)block_minmax_f<1>(fn, sh);
        mx = (double)block_minmax_f<2>(fx, sh);
    } else {
        double acc = 0.0, dn = 1e300, dx = -1e300;
        for (int a = ps.lo + threadIdx.x; a < ps.hi; a += blockDim.x) {
            const double z = (double)h[ps.base + (size_t)a * ps.stride];
            acc += z;
            dn = fmin(dn, z);
            dx = fmax(dx, z);
        }
        sum = block_reduce<0>(acc, sh);
        mn = block_reduce<1>(dn, sh);
        mx = block_reduce<2>(dx, sh);
    }
    if (threadIdx.x == 0) {
        double* o = ppart + 4 * (size_t)item;
        o[0] = sum;
        o[1] = mn;
        o[2] = mx;
    }
}

// Mean of a profile from its segments' pass-1 sums (fixed order).
__device__ __forceinline__ double profile_mean(const double* ppart, int prof, int L) {
    double s = 0.0;
    for (int seg = 0; seg < kRzSegments; ++seg) s += __ldcg(ppart + 4 * ((size_t)prof * kRzSegments + seg));
    return s / (double)L;
}

// Pass 2 of a profile segment: sum of |z - profile mean| (FP32 maps:
// double-float, each deviation formed exactly).
template <typename T>
__device__ void profile_seg2(const RoughJob* __restrict__ jobs, int item, int per_job, double* ppart, double* sh) {
    const int j = item / (per_job * kRzSegments), rem = item - j * per_job * kRzSegments;
    const int q = rem / kRzSegments, seg = rem - q * kRzSegments;
    const RoughJob jb = jobs[j];
    const ProfileSeg ps = profile_seg(jb, q, seg);
    if (!ps.valid) return;
    const T* h = reinterpret_cast<const T*>(jb.h);
    const double mu = profile_mean(ppart, j * per_job + q, ps.L);
    double dev;
    if constexpr (sizeof(T) == 4) {
        const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
        float2 w = make_float2(0.f, 0.f);
        for (int a = ps.lo + threadIdx.x; a < ps.hi; a += blockDim.x) {
            float d, e, dh, dl;
            two_sum((float)h[ps.base + (size_t)a * ps.stride], -mu_hi, &d, &e);
            two_sum(d, e - mu_lo, &dh, &dl);  // z - mu as a normalised pair: its sign is dh's
            w = df_add(w, dh < 0.f ? make_float2(-dh, -dl) : make_float2(dh, dl));
        }
        dev = block_sum_df(w, sh);
    } else {
        double w = 0.0;
        for (int a = ps.lo + threadIdx.x; a < ps.hi; a += blockDim.x)
            w += fabs((double)h[ps.base + (size_t)a * ps.stride] - mu);
        dev = block_reduce<0>(w, sh);
    }
    if (threadIdx.x == 0) ppart[4 * (size_t)item + 3] = dev;
}

// Profile results of job j (the block finalising the job; a thread per
// profile, its segments combined in order).
__device__ void finalize_profiles(const RoughJob& jb, int j, int per_job, const double* ppart) {
    fsm_roughness_out* out = jb.out;
    for (int q = threadIdx.x; q < jb.n_rows + jb.n_cols; q += blockDim.x) {
        const ProfileSeg ps = profile_seg(jb, q, 0);
        const int prof = j * per_job + q;
        double dev = 0.0, rz = 0.0;
        for (int seg = 0; seg < kRzSegments; ++seg) {
            const double* o = ppart + 4 * ((size_t)prof * kRzSegments + seg);
            dev += __ldcg(o + 3);
            rz += __ldcg(o + 2) - __ldcg(o + 1);
        }
        const double ra = dev / (double)ps.L;
        const double rzv = ps.L >= kRzSegments ? rz / (double)kRzSegments : __longlong_as_double(0x7ff8000000000000ll);
        if (ps.row) {
            out->row_index[ps.r] = ps.fixed;
            out->Ra_row[ps.r] = ra;
            out->Rz_row[ps.r] = rzv;
        } else {
            out->col_index[ps.r] = ps.fixed;
            out->Ra_col[ps.r] = ra;
            out->Rz_col[ps.r] = rzv;
        }
    }
}


// End of a pass-2 item of job j: the block completing the job's last item
// (chunks and profile segments) combines it.
__device__ __forceinline__ void finish2(const RoughJob* __restrict__ jobs, int n_jobs,
                                        const int* __restrict__ chunk_base, const double* part, const double* part2,
                                        void* sync, int total_chunks, int per_job, int j, double* sh) {
    const RoughSync rs = rough_sync(sync, n_jobs);
    const int items = chunk_base[j + 1] - chunk_base[j] + per_job * kRzSegments;
    if (last_chunk_block(rs.done2, j, items))
        finalize_job(jobs, chunk_base, part, part2, j, __ldcg(rs.mean + j), per_job,
                     part + 7 * (size_t)total_chunks, sh);
}

// Pass-2 items past the chunks are profile segments; true if b was one.
template <typename T>
__device__ __forceinline__ bool rough2_profile(const RoughJob* __restrict__ jobs, int n_jobs,
                                               const int* __restrict__ chunk_base, const double* part,
                                               const double* part2, void* sync, int total_chunks, int per_job, int b,
                                               double* sh) {
    if (b < total_chunks) return false;
    const int it = b - total_chunks;
    profile_seg2<T>(jobs, it, per_job, const_cast<double*>(part) + 7 * (size_t)total_chunks, sh);
    finish2(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, it / (per_job * kRzSegments), sh);
    return true;
}

// Pass 2: per chunk sums of |d|, d^2, d^3, d^4 about the job mean -> part2[b*4 + a]
template <typename T>
__device__ __forceinline__ void rough2_item(const RoughJob* __restrict__ jobs, int n_jobs,
                                            const int* __restrict__ chunk_base, const double* part, double* part2,
                                            void* sync, int total_chunks, int per_job, int b, double* sh) {
    if (rough2_profile<T>(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, b, sh)) return;
    const int j = find_job(chunk_base, n_jobs, b);
    const RoughJob jb = jobs[j];
    const RoughSync rs = rough_sync(sync, n_jobs);
    const double mu = rs.mean[j];
    size_t lo, hi;
    chunk_range<T>(jb, b - chunk_base[j], &lo, &hi);
    const T* h = reinterpret_cast<const T*>(jb.h);
    // |d|, d^2, d^3, d^4 of d = z - mu (one FP64 subtraction, split into a
    // float pair) in double-float on the FP32 pipes
    float2 v[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 2
    for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const float2 d = split_double((double)h[i] - mu);
        const float2 d2 = df_mul(d, d);
        v[0] = df_add(v[0], d.x < 0.f ? make_float2(-d.x, -d.y) : d);
        v[1] = df_add(v[1], d2);
        v[2] = df_add(v[2], df_mul(d2, d));
        v[3] = df_add(v[3], df_mul(d2, d2));
    }
    double vs[4];
    block_sum_df4(v, sh, vs);
    if (threadIdx.x == 0) {
        double* o = part2 + 4 * (size_t)b;
        o[0] = vs[0]; o[1] = vs[1]; o[2] = vs[2]; o[3] = vs[3];
    }
    // the block that finishes a job's last item combines the job
    finish2(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, j, sh);
}

// FP32 maps: the same two passes with 16-byte loads and no FP64 arithmetic
// per cell or per chunk: per-cell terms in FP32, summed in FP32 over 32
// cells (relative error of a leaf <= 32 u ~ 2e-6, far inside the FP32 path's
// 1e-4 target), the leaves and the block sums kept as double-float pairs.
// Pass 1 sums z - ref about the map's first cell, so its leaves carry
// deviations only; min and max are exact in FP32. The mean is used as a
// float pair so the deviations keep full FP32 precision. (FP64 maps take
// their cells as float pairs and double-float terms throughout.)
__device__ __forceinline__ bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

__device__ __forceinline__ void rough1_f32_item(const RoughJob* __restrict__ jobs, int n_jobs,
                                                const int* __restrict__ chunk_base, double* part, int total_chunks,
                                                int per_job, void* sync, int b, double* sh) {
    if (b >= total_chunks) {  // items past the chunks are profile segments
        profile_seg1<float>(jobs, b - total_chunks, per_job, part + 7 * (size_t)total_chunks, sh);
        return;
    }
    const int j = find_job(chunk_base, n_jobs, b);
    const RoughJob jb = jobs[j];
    size_t lo, hi;
    chunk_range<float>(jb, b - chunk_base[j], &lo, &hi);
    const float* h = reinterpret_cast<const float*>(jb.h);
    const float ref = __ldg(h);
    float2 s = make_float2(0.f, 0.f);  // sum of z - ref
    float mn = 3.0e38f, mx = -3.0e38f;
    if (aligned16(h)) {
        const size_t v0 = lo >> 2, v1 = hi >> 2;  // lo is a multiple of 4
        const float4* h4 = reinterpret_cast<const float4*>(h);
        size_t v = v0 + threadIdx.x;
        while (v < v1) {
            float leaf = 0.f;
#pragma unroll
            for (int r = 0; r < 8; ++r, v += blockDim.x) {
                if (v < v1) {
                    const float4 q = __ldg(h4 + v);
                    leaf += ((q.x - ref) + (q.y - ref)) + ((q.z - ref) + (q.w - ref));
                    mn = fminf(mn, fminf(fminf(q.x, q.y), fminf(q.z, q.w)));
                    mx = fmaxf(mx, fmaxf(fmaxf(q.x, q.y), fmaxf(q.z, q.w)));
                }
            }
            s = df_add(s, make_float2(leaf, 0.f));
        }
        for (size_t i = (v1 << 2) + threadIdx.x; i < hi; i += blockDim.x) {
            const float z = h[i];
            s = df_add(s, make_float2(z - ref, 0.f));
            mn = fminf(mn, z);
            mx = fmaxf(mx, z);
        }
    } else {
        for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float z = h[i];
            s = df_add(s, make_float2(z - ref, 0.f));
            mn = fminf(mn, z);
            mx = fmaxf(mx, z);
        }
    }
    const double sum = block_sum_df(s, sh);
    mn = block_minmax_f<1>(mn, sh);
    mx = block_minmax_f<2>(mx, sh);
    if (threadIdx.x == 0) {
        part[3 * (size_t)b] = sum;
        part[3 * (size_t)b + 1] = (double)mn;
        part[3 * (size_t)b + 2] = (double)mx;
    }
    job_mean_if_last(jobs, chunk_base, part, n_jobs, j, sync, (double)ref, sh);
}

__device__ __forceinline__ void dev_terms(float z, float mu_hi, float mu_lo, float* a) {
    const float d = (z - mu_hi) - mu_lo;
    const float d2 = d * d;
    a[0] += fabsf(d);
    a[1] += d2;
    a[2] = fmaf(d2, d, a[2]);
    a[3] = fmaf(d2, d2, a[3]);
}

__device__ __forceinline__ void rough2_f32_item(const RoughJob* __restrict__ jobs, int n_jobs,
                                                const int* __restrict__ chunk_base, const double* part, double* part2,
                                                void* sync, int total_chunks, int per_job, int b, double* sh) {
    if (rough2_profile<float>(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, b, sh)) return;
    const int j = find_job(chunk_base, n_jobs, b);
    const RoughJob jb = jobs[j];
    const RoughSync rs = rough_sync(sync, n_jobs);
    const double mu = rs.mean[j];
    const float mu_hi = (float)mu, mu_lo = (float)(mu - (double)mu_hi);
    size_t lo, hi;
    chunk_range<float>(jb, b - chunk_base[j], &lo, &hi);
    const float* h = reinterpret_cast<const float*>(jb.h);
    float2 v[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (aligned16(h)) {
        const size_t v0 = lo >> 2, v1 = hi >> 2;
        const float4* h4 = reinterpret_cast<const float4*>(h);
        size_t q = v0 + threadIdx.x;
        while (q < v1) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int r = 0; r < 8; ++r, q += blockDim.x) {
                if (q < v1) {
                    const float4 z = __ldg(h4 + q);
                    dev_terms(z.x, mu_hi, mu_lo, a);
                    dev_terms(z.y, mu_hi, mu_lo, a);
                    dev_terms(z.z, mu_hi, mu_lo, a);
                    dev_terms(z.w, mu_hi, mu_lo, a);
                }
            }
            for (int k = 0; k < 4; ++k) v[k] = df_add(v[k], make_float2(a[k], 0.f));
        }
        for (size_t i = (v1 << 2) + threadIdx.x; i < hi; i += blockDim.x) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            dev_terms(h[i], mu_hi, mu_lo, a);
            for (int k = 0; k < 4; ++k) v[k] = df_add(v[k], make_float2(a[k], 0.f));
        }
    } else {
        for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            float a[4] = {0.f, 0.f, 0.f, 0.f};
            dev_terms(h[i], mu_hi, mu_lo, a);
            for (int k = 0; k < 4; ++k) v[k] = df_add(v[k], make_float2(a[k], 0.f));
        }
    }
    double vs[4];
    block_sum_df4(v, sh, vs);
    if (threadIdx.x == 0) {
        double* o = part2 + 4 * (size_t)b;
        o[0] = vs[0]; o[1] = vs[1]; o[2] = vs[2]; o[3] = vs[3];
    }
    // the block that finishes a job's last item combines the job
    finish2(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, j, sh);
}

// Persistent roughness passes: blocks walk the items (pass 1: profiles, then chunks)
// in a grid stride; partial results are stored per chunk, so the combine
// order does not depend on which block took which chunk.
template <typename T>
__global__ void __launch_bounds__(256, kRoughBlocksPerSm) rough1_kernel(const RoughJob* __restrict__ jobs, int n_jobs,
                                                     const int* __restrict__ chunk_base, double* part,
                                                     int total_chunks, int per_job, void* sync, int n_items) {
    __shared__ double sh[32];
    const int n_prof = n_items - total_chunks;  // profile segments first
    for (int b = blockIdx.x; b < n_items; b += gridDim.x) {
        const int item = b < n_prof ? total_chunks + b : b - n_prof;
        rough1_item<T>(jobs, n_jobs, chunk_base, part, total_chunks, per_job, sync, item, sh);
    }
}
__global__ void __launch_bounds__(256, kRoughBlocksPerSm) rough1_f32_kernel(const RoughJob* __restrict__ jobs, int n_jobs,
                                                         const int* __restrict__ chunk_base, double* part,
                                                         int total_chunks, int per_job, void* sync, int n_items) {
    __shared__ double sh[32];
    const int n_prof = n_items - total_chunks;  // profile segments first
    for (int b = blockIdx.x; b < n_items; b += gridDim.x) {
        const int item = b < n_prof ? total_chunks + b : b - n_prof;
        rough1_f32_item(jobs, n_jobs, chunk_base, part, total_chunks, per_job, sync, item, sh);
    }
}
// Pass 2 walks the profile segments first, then the chunks.
template <typename T>
__global__ void __launch_bounds__(256, kRoughBlocksPerSm) rough2_kernel(const RoughJob* __restrict__ jobs, int n_jobs,
                                                     const int* __restrict__ chunk_base, const double* part,
                                                     double* part2, void* sync, int total_chunks, int per_job,
                                                     int n_items) {
    __shared__ double sh[128];
    const int n_prof = n_items - total_chunks;
    for (int b = blockIdx.x; b < n_items; b += gridDim.x) {
        const int item = b < n_prof ? total_chunks + b : b - n_prof;
        rough2_item<T>(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, item, sh);
    }
}
__global__ void __launch_bounds__(256, kRoughBlocksPerSm) rough2_f32_kernel(const RoughJob* __restrict__ jobs, int n_jobs,
                                                         const int* __restrict__ chunk_base, const double* part,
                                                         double* part2, void* sync, int total_chunks, int per_job,
                                                         int n_items) {
    __shared__ double sh[128];
    const int n_prof = n_items - total_chunks;
    for (int b = blockIdx.x; b < n_items; b += gridDim.x) {
        const int item = b < n_prof ? total_chunks + b : b - n_prof;
        rough2_f32_item(jobs, n_jobs, chunk_base, part, part2, sync, total_chunks, per_job, item, sh);
    }
}

// ===========================================================================
// Moment partials of a map or of one band of a map (a map split into row
// bands over several devices combines its roughness from these): chunk b of
// the map gives [n, sum d, min z, max z, sum |d|, sum d^2, sum d^3, sum d^4]
// with d = z - about; a single block then adds the chunks in chunk order.
// FP64 maps: FP64; FP32 maps: each d formed as a float pair, the terms in
// double-float on the FP32 pipes.
// ===========================================================================
template <typename T>
__global__ void __launch_bounds__(256) moment_chunks_kernel(const T* __restrict__ h, size_t n, double about,
                                                            double* __restrict__ part) {
    __shared__ double sh[32];
    const size_t lo = (size_t)blockIdx.x * kChunk, hi = lo + kChunk < n ? lo + kChunk : n;
    double r[8];
    if constexpr (sizeof(T) == 4) {
        const float a_hi = (float)about, a_lo = (float)(about - (double)a_hi);
        float2 acc[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float mn = 3.0e38f, mx = -3.0e38f;
        for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const float z = (float)h[i];
            float d, e, dh, dl;
            two_sum(z, -a_hi, &d, &e);
            two_sum(d, e - a_lo, &dh, &dl);  // z - about as a normalised pair
            const float d2 = dh * dh, d3 = d2 * dh;
            acc[0] = df_add(acc[0], make_float2(dh, dl));
            acc[1] = df_add(acc[1], dh < 0.f ? make_float2(-dh, -dl) : make_float2(dh, dl));
            acc[2] = df_add(acc[2], make_float2(d2, fmaf(dh, dh, -d2) + 2.f * dh * dl));
            acc[3] = df_add(acc[3], make_float2(d3, 0.f));
            acc[4] = df_add(acc[4], make_float2(d2 * d2, 0.f));
            mn = fminf(mn, z);
            mx = fmaxf(mx, z);
        }
        r[1] = block_sum_df(acc[0], sh);
        r[4] = block_sum_df(acc[1], sh);
        r[5] = block_sum_df(acc[2], sh);
        r[6] = block_sum_df(acc[3], sh);
        r[7] = block_sum_df(acc[4], sh);
        r[2] = (double)block_minmax_f<1>(mn, sh);
        r[3] = (double)block_minmax_f<2>(mx, sh);
    } else {
        double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, mn = 1e300, mx = -1e300;
        for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double z = (double)h[i];
            const double d = z - about, d2 = d * d;
            a[0] += d;
            a[1] += fabs(d);
            a[2] += d2;
            a[3] += d2 * d;
            a[4] += d2 * d2;
            mn = fmin(mn, z);
            mx = fmax(mx, z);
        }
        r[1] = block_reduce<0>(a[0], sh);
        r[4] = block_reduce<0>(a[1], sh);
        r[5] = block_reduce<0>(a[2], sh);
        r[6] = block_reduce<0>(a[3], sh);
        r[7] = block_reduce<0>(a[4], sh);
        r[2] = block_reduce<1>(mn, sh);
        r[3] = block_reduce<2>(mx, sh);
    }
    if (threadIdx.x == 0) {
        r[0] = (double)(hi - lo);
        for (int k = 0; k < 8; ++k) part[8 * (size_t)blockIdx.x + k] = r[k];
    }
}

__global__ void __launch_bounds__(256) moment_combine_kernel(const double* __restrict__ part, int chunks,
                                                             double* __restrict__ out) {
    __shared__ double sh[32];
    double v[8] = {0.0, 0.0, 1e300, -1e300, 0.0, 0.0, 0.0, 0.0};
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
        const double* p = part + 8 * (size_t)c;
        v[0] += p[0]; v[1] += p[1]; v[4] += p[4]; v[5] += p[5]; v[6] += p[6]; v[7] += p[7];
        v[2] = fmin(v[2], p[2]);
        v[3] = fmax(v[3], p[3]);
    }
    double r[8];
    for (int k = 0; k < 8; ++k) r[k] = k == 2 ? block_reduce<1>(v[k], sh) : k == 3 ? block_reduce<2>(v[k], sh)
                                                                                   : block_reduce<0>(v[k], sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 8; ++k) out[k] = r[k];
}

size_t moment_ws_bytes(size_t n) { return 8 * sizeof(double) * ((n + kChunk - 1) / kChunk); }

cudaError_t launch_moments(int precision, const void* d_h, size_t n, double about, double* d_ws, double* d_out,
                           cudaStream_t st) {
    const int chunks = (int)((n + kChunk - 1) / kChunk);
    if (precision == 0)
        moment_chunks_kernel<double><<<chunks, 256, 0, st>>>((const double*)d_h, n, about, d_ws);
    else
        moment_chunks_kernel<float><<<chunks, 256, 0, st>>>((const float*)d_h, n, about, d_ws);
    moment_combine_kernel<<<1, 256, 0, st>>>(d_ws, chunks, d_out);
    return cudaGetLastError();
}

// ===========================================================================
// Launchers (called by the C ABI layer)
// ===========================================================================
// ---------------------------------------------------------------------------
// Trajectory map (Section 3.1). The tool reference moves in a horizontal
// plane, so the height of edge point (K, j) at step s depends on the spindle
// phase m = s mod S alone: the lowest point of each edge is tabulated once
// per (m, K) -- one warp each, a lexicographic (z, j) minimum -- and every
// time step then evaluates one FP64 pose per tooth, through the same pose
// arithmetic as the FP64 map.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) traj_argmin_kernel(const Surface* __restrict__ sp, int32_t* __restrict__ jmin) {
    const Surface& sf = *sp;
    const int N = sf.n_teeth, E = sf.E, NE = N * E;
    const long long wi = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (wi >= (long long)sf.S * N) return;
    const int lane = threadIdx.x & 31;
    const int m = (int)(wi / N), K = (int)(wi - (long long)m * N);
    const double2 cs = sf.ph64[m];
    const double zr = sf.z_ref;
    const double* uz = sf.tool64 + 2 * NE + K * E;
    const double* vz = sf.tool64 + 5 * NE + K * E;
    const double* wz = sf.tool64 + 8 * NE + K * E;
    double bz = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    int bj = 0x7fffffff;
    for (int j = lane; j < E; j += 32) {
        const double z = __dadd_rn(zr, __fma_rn(cs.x, uz[j], __fma_rn(cs.y, vz[j], wz[j])));
        if (z < bz) {
            bz = z;
            bj = j;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const double oz = __shfl_xor_sync(0xffffffffu, bz, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (oz < bz || (oz == bz && oj < bj)) {
            bz = oz;
            bj = oj;
        }
    }
    if (lane == 0) jmin[wi] = bj;
}

__global__ void __launch_bounds__(256) traj_record_kernel(const Surface* __restrict__ sp,
                                                          const int32_t* __restrict__ jmin,
                                                          fsm_traj_point* __restrict__ out, int n_steps) {
    const Surface& sf = *sp;
    const int N = sf.n_teeth, E = sf.E, S = sf.S, NE = N * E, spp = sf.steps_per_pass;
    const double zr = sf.z_ref;
    // one thread per time step writes its n_teeth consecutive records
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_steps; s += gridDim.x * blockDim.x) {
        const int p = s / spp;
        const int m = s % S;
        const double xc = path_x(sf, p, s - p * spp), yc = path_y(sf, p, s - p * spp);
        const double2 cs = __ldg(sf.ph64 + m);
        fsm_traj_point* o = out + (size_t)s * N;
        for (int K = 0; K < N; ++K) {
            const int j = __ldg(jmin + m * N + K);
            const Vec9 v = load_vec9(sf.tool64, NE, K * E + j);
            const Pose64 P = pose64(v, cs, xc, yc, zr);
            double2* d = reinterpret_cast<double2*>(o + K);
            d[0] = make_double2(P.x, P.y);
            d[1] = make_double2(P.z, __hiloint2double(K, j));  // (j, tooth) as two little-endian int32
        }
    }
}

cudaError_t launch_trajectory(const Surface* d_surf, int S, int n_teeth, long long n_records, int32_t* d_jmin,
                              fsm_traj_point* d_out, cudaStream_t st) {
    const long long warps = (long long)S * n_teeth;
    traj_argmin_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(d_surf, d_jmin);
    const int n_steps = (int)(n_records / n_teeth);  // total steps < 2^31
    if (n_steps > 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int blocks = (int)std::min<long long>((n_steps + 255) / 256, (long long)sms * 8);
        traj_record_kernel<<<blocks, 256, 0, st>>>(d_surf, d_jmin, d_out, n_steps);
    }
    return cudaGetLastError();
}

cudaError_t launch_plan(Surface* d_surfs, int n, const Surface* one, int max_work, int sm_count, cudaStream_t st) {
    Surface dummy;
    if (one) dummy = *one;
    else memset(&dummy, 0, sizeof dummy);
    // The FP64 tables (edge points, and the phase table: tens of thousands
    // of phases at fine time steps) are built with FP64 transcendentals on
    // GB300's 1/64-rate FP64 pipe, so a surface's work is spread over as many
    // SMs as it fills: small blocks of 64 threads, about one item each, while
    // the grid stays within ~16 blocks per SM; large batches give each
    // surface one block (the 5 mm ball raster: 107 blocks, 34 us against
    // 39 us for 27 blocks of 256).
    constexpr int kPlanThreads = 64;
    if (one) max_work = one->n_teeth * one->E + one->S;
    const int want = max(1, min(kPlanParts, (max_work + kPlanThreads - 1) / kPlanThreads));
    const int fit = max(1, 16 * max(sm_count, 1) / max(n, 1));
    const int parts = one ? want : min(want, fit);
    plan_kernel<<<dim3(n, parts), kPlanThreads, 0, st>>>(d_surfs, n, dummy, one ? 1 : 0);
    plan_finish_kernel<<<n, 256, 0, st>>>(d_surfs, n, parts);
    return cudaGetLastError();
}

size_t sweep_smem_bytes(int precision, int tile_x, int tile_y, int threads) {
    const size_t cell = precision == 0 ? 8 : 4;
    return sweep_scratch_bytes(precision, threads) + cell * (size_t)tile_x * (size_t)tile_y;
}

size_t sweep_static_bytes() { return sizeof(TileShared) + 2 * sizeof(int); }

cudaError_t launch_sweep_shaped(int precision, const Surface* d_surfs, int n_surf,
                                const int* d_tile_base, int total_tiles, int* d_queue,
                                long long* d_counters, int grid, int threads, size_t smem,
                                cudaStream_t st, bool phase_form, bool tilt) {
    // counting, the FP32 phase form and tilted feeds are separate
    // instantiations: without them the counters are dead code and the item
    // loop has the SM to itself
    if (tilt) {
        if (precision == 0 && d_counters)
            sweep_kernel<true, true, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                               total_tiles, d_queue, d_counters);
        else if (precision == 0)
            sweep_kernel<true, false, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                                total_tiles, d_queue, nullptr);
        else if (d_counters)
            sweep_kernel<false, true, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                                total_tiles, d_queue, d_counters);
        else
            sweep_kernel<false, false, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                                 total_tiles, d_queue, nullptr);
    } else if (precision == 0 && phase_form) {
        if (d_counters)
            sweep_kernel<true, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base, total_tiles,
                                                                        d_queue, d_counters);
        else
            sweep_kernel<true, false, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                         total_tiles, d_queue, nullptr);
    } else if (precision == 0) {
        if (d_counters)
            sweep_kernel<true, true, false><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base, total_tiles,
                                                                         d_queue, d_counters);
        else
            sweep_kernel<true, false, false><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                          total_tiles, d_queue, nullptr);
    } else if (phase_form) {
        if (d_counters)
            sweep_kernel<false, true, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base, total_tiles,
                                                                         d_queue, d_counters);
        else
            sweep_kernel<false, false, true><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                          total_tiles, d_queue, nullptr);
    } else {
        if (d_counters)
            sweep_kernel<false, true, false><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                          total_tiles, d_queue, d_counters);
        else
            sweep_kernel<false, false, false><<<grid, threads, smem, st>>>(d_surfs, n_surf, d_tile_base,
                                                                           total_tiles, d_queue, nullptr);
    }
    return cudaGetLastError();
}

// Allow the sweep kernels the device's whole opt-in shared memory; called once
// per context with its device current (not a stream operation).
template <typename K>
static cudaError_t allow_dynamic_smem(K kernel, size_t max_bytes) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    const size_t dyn = max_bytes > a.sharedSizeBytes ? max_bytes - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t sweep_allow_smem(size_t max_bytes) {
    cudaError_t e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, true, false>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, false, false>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, true, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, false, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<false, true, false>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<false, false, false>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<false, true, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<false, false, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, true, true, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<true, false, true, true>, max_bytes)) != cudaSuccess) return e;
    if ((e = allow_dynamic_smem(sweep_kernel<false, true, true, true>, max_bytes)) != cudaSuccess) return e;
    return allow_dynamic_smem(sweep_kernel<false, false, true, true>, max_bytes);
}

// Resident CTAs per SM: the smallest over the instantiations of a precision.
int sweep_blocks_per_sm(int precision, int threads, size_t smem) {
    int r[6] = {0, 0, 0, 0, 0, 0};
    cudaError_t e[6];
    if (precision == 0) {
        e[0] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 0, sweep_kernel<true, true, false>, threads, smem);
        e[1] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 1, sweep_kernel<true, false, false>, threads, smem);
        e[2] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 2, sweep_kernel<true, true, true>, threads, smem);
        e[3] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 3, sweep_kernel<true, false, true>, threads, smem);
        e[4] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 4, sweep_kernel<true, true, true, true>, threads,
                                                             smem);
        e[5] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 5, sweep_kernel<true, false, true, true>, threads,
                                                             smem);
    } else {
        e[0] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 0, sweep_kernel<false, true, false>, threads, smem);
        e[1] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 1, sweep_kernel<false, false, false>, threads, smem);
        e[2] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 2, sweep_kernel<false, true, true>, threads, smem);
        e[3] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 3, sweep_kernel<false, false, true>, threads, smem);
        e[4] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 4, sweep_kernel<false, true, true, true>, threads,
                                                             smem);
        e[5] = cudaOccupancyMaxActiveBlocksPerMultiprocessor(r + 5, sweep_kernel<false, false, true, true>,
                                                             threads, smem);
    }
    int b = 1 << 20;
    for (int k = 0; k < 6; ++k) {
        if (e[k] != cudaSuccess) return 0;
        b = min(b, r[k]);
    }
    return b;
}

__global__ void rough_setup_one_kernel(RoughJob jb, int chunks, RoughJob* d_job, int* d_base) {
    if (threadIdx.x == 0) {
        *d_job = jb;
        d_base[0] = 0;
        d_base[1] = chunks;
    }
}

cudaError_t launch_roughness_one(int precision, const RoughJob& jb, char* d_ws, cudaStream_t st) {
    const int chunks = (int)((jb.n + kChunk - 1) / kChunk);
    RoughJob* d_job = (RoughJob*)d_ws;
    int* d_base = (int*)(d_ws + 256);
    void* d_sync = d_ws + 320;  // rough_sync_bytes(1) = 16
    double* d_part = (double*)(d_ws + 512);
    rough_setup_one_kernel<<<1, 32, 0, st>>>(jb, chunks, d_job, d_base);
    return launch_roughness_jobs(precision, d_job, 1, d_base, chunks, jb.n_rows + jb.n_cols, d_part, d_sync, st);
}

size_t rough_part_doubles(int total_chunks, int n_jobs, int max_profiles) {
    return 7 * (size_t)total_chunks + 4 * (size_t)kRzSegments * (size_t)n_jobs * (size_t)max_profiles;
}

size_t roughness_one_ws_bytes(size_t n) {
    const size_t chunks = (n + kChunk - 1) / kChunk;
    return 512 + sizeof(double) * rough_part_doubles((int)chunks, 1, 2 * FSM_MAX_PROFILES);
}

size_t rough_sync_bytes(int n_jobs) { return ((8 * (size_t)n_jobs + 7) & ~(size_t)7) + 8 * (size_t)n_jobs; }

cudaError_t launch_roughness_jobs(int precision, const RoughJob* d_jobs, int n_jobs, const int* d_chunk_base,
                                  int total_chunks, int max_profiles, double* d_part, void* d_sync,
                                  cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    double* part2 = d_part + 3 * (size_t)total_chunks;
    cudaError_t e = cudaMemsetAsync(d_sync, 0, rough_sync_bytes(n_jobs), st);
    if (e != cudaSuccess) return e;
    // pass 1 (profile segments, then the chunks; each job's last chunk block
    // stores the mean), pass 2 (the same items; each job's last block
    // combines it); both persistent, kRoughBlocksPerSm blocks per SM
    const int per_job = max(max_profiles, 1);
    const int items = total_chunks + n_jobs * per_job * kRzSegments;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int g = std::min(items, kRoughBlocksPerSm * sms);
    if (precision == 0) {
        rough1_kernel<double><<<g, 256, 0, st>>>(d_jobs, n_jobs, d_chunk_base, d_part, total_chunks, per_job, d_sync,
                                                items);
        rough2_kernel<double><<<g, 256, 0, st>>>(d_jobs, n_jobs, d_chunk_base, d_part, part2, d_sync, total_chunks,
                                                per_job, items);
    } else {
        rough1_f32_kernel<<<g, 256, 0, st>>>(d_jobs, n_jobs, d_chunk_base, d_part, total_chunks, per_job, d_sync,
                                            items);
        rough2_f32_kernel<<<g, 256, 0, st>>>(d_jobs, n_jobs, d_chunk_base, d_part, part2, d_sync, total_chunks,
                                            per_job, items);
    }
    return cudaGetLastError();
}

}  // namespace fsm

// ===========================================================================
// Allocation-free roughness: the same launches as fsm_roughness with the
// scratch (job record, chunk prefix, per-chunk partials) in a fixed device
// array, for callers that may not allocate device memory while running.
// ===========================================================================
namespace fsm {

constexpr size_t kNoAllocMaxCells = (size_t)1 << 29;
constexpr size_t kNoAllocChunks = (kNoAllocMaxCells + kChunk - 1) / kChunk;
constexpr size_t kNoAllocBytes =
    512 + sizeof(double) * (7 * kNoAllocChunks + 4 * 5 * 2 * FSM_MAX_PROFILES);  // about 0.9 MiB

// One per device that loads the library, kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array on ctx's device, looked up on the context's
// first call with that device current and kept in the context (in host code
// the symbol names a host-side stand-in, not memory the GPU can use). A
// context lives inside one CUDA primary context of its device: after a
// cudaDeviceReset the library's contexts must be recreated, which also
// repeats this look-up.
static char* noalloc_scratch(fsm_ctx* ctx, cudaError_t* err) {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->noalloc_scratch) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        ctx->noalloc_scratch = (char*)p;
    }
    *err = cudaSuccess;
    return ctx->noalloc_scratch;
}

}  // namespace fsm

extern "C" fsm_status fsm_roughness_noalloc(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx,
                                            int32_t ny, int32_t n_rows, int32_t n_cols,
                                            fsm_roughness_out* d_out, void* stream) {
    using namespace fsm;
    if (!ctx || !d_heights || !d_out) return fail(FSM_E_INVALID, "ctx/d_heights/d_out is NULL");
    if (precision != FSM_FP64 && precision != FSM_FP32) return fail(FSM_E_INVALID, "unknown precision");
    if (nx < 1 || ny < 1) return fail(FSM_E_INVALID, "nx, ny must be >= 1");
    if (n_rows < 0 || n_cols < 0 || n_rows > FSM_MAX_PROFILES || n_cols > FSM_MAX_PROFILES)
        return fail(FSM_E_INVALID, "0 <= n_rows, n_cols <= 16");
    const size_t n = (size_t)nx * (size_t)ny;
    if (n > kNoAllocMaxCells)
        return fail(FSM_E_INVALID, "fsm_roughness_noalloc handles at most 2^29 cells (" +
                                       std::to_string(kNoAllocMaxCells) + "); this map has " + std::to_string(n));
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    char* ws = noalloc_scratch(ctx, &e);
    if (!ws) return cuda_fail(e, "cudaGetSymbolAddress (no-alloc scratch)");
    RoughJob jb;
    jb.h = d_heights;
    jb.n = n;
    jb.nx = nx;
    jb.ny = ny;
    jb.n_rows = n_rows;
    jb.n_cols = n_cols;
    jb.out = d_out;
    if ((e = launch_roughness_one(precision, jb, ws, (cudaStream_t)stream)) != cudaSuccess)
        return cuda_fail(e, "roughness kernels (no-alloc)");
    return FSM_OK;
}
