// fsm_api.cpp -- C ABI of the FSM surface generator: validation, plan
// layout and launches. No arithmetic of the method runs here; the host only
// copies descriptors into per-surface plans, sizes stream-ordered scratch and
// enqueues kernels.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fsm.h"
#include "fsm_host.h"
#include "fsm_internal.h"

using fsm::Surface;

namespace {
thread_local std::string g_err;
}  // namespace

namespace fsm {

fsm_status fail(fsm_status st, const std::string& msg) {
    g_err = msg;
    return st;
}

fsm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(FSM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static bool finite(double v) { return isfinite(v) != 0; }

static int64_t steps_per_rev(double step_deg) {
    if (!(step_deg > 0.0) || !finite(step_deg)) return -1;
    const double r = 360.0 / step_deg;
    const int64_t S = (int64_t)llround(r);
    if (S < 1 || fabs(r - (double)S) > 1e-9 * (double)S || S > (1 << 22)) return -1;
    return S;
}

static fsm_status check_tool(const fsm_tool_desc* t) {
    if (!t) return fail(FSM_E_INVALID, "tool descriptor is NULL");
    if (t->kind != FSM_TOOL_FLAT && t->kind != FSM_TOOL_BALL && t->kind != FSM_TOOL_INSERT &&
        t->kind != FSM_TOOL_TORUS)
        return fail(FSM_E_INVALID, "unknown tool kind");
    if (t->kind == FSM_TOOL_TORUS &&
        !(t->corner_radius > 0.0 && t->corner_radius <= 0.5 * t->diameter && finite(t->corner_radius)))
        return fail(FSM_E_INVALID, "corner_radius must be in (0, D/2]");
    if (t->kind == FSM_TOOL_INSERT) {
        if (!(t->insert_radius > 0.0) || !finite(t->insert_radius))
            return fail(FSM_E_INVALID, "insert_radius must be > 0");
        const double v[] = {t->rake_f_deg, t->rake_p_deg, t->eps_r_mm, t->eps_a_mm};
        for (double x : v)
            if (!finite(x)) return fail(FSM_E_INVALID, "non-finite insert parameter");
        if (fabs(t->rake_f_deg) >= 80.0 || fabs(t->rake_p_deg) >= 80.0) return fail(FSM_E_INVALID, "|rake| < 80");
    }
    if (t->n_teeth < 1 || t->n_teeth > FSM_MAX_TEETH) return fail(FSM_E_INVALID, "n_teeth must be 1..16");
    if (t->n_edge < 2) return fail(FSM_E_INVALID, "n_edge must be >= 2");
    const bool has_end = t->kind == FSM_TOOL_FLAT || t->kind == FSM_TOOL_TORUS;
    if (has_end && (t->n_end < 0 || t->n_end == 1)) return fail(FSM_E_INVALID, "n_end must be 0 or >= 2");
    if (!has_end && t->n_end != 0) return fail(FSM_E_INVALID, "only flat and torus ends have n_end > 0");
    if ((int64_t)t->n_teeth * (t->n_edge + t->n_end) > (1 << 22))
        return fail(FSM_E_INVALID, "too many edge points");
    if (!(t->diameter > 0.0) || !finite(t->diameter)) return fail(FSM_E_INVALID, "diameter must be > 0");
    if (!(t->runout_mm >= 0.0) || !finite(t->runout_mm) || !finite(t->runout_phase_deg))
        return fail(FSM_E_INVALID, "runout must be finite and >= 0");
    for (int k = 0; k < t->n_teeth; ++k)
        if (!finite(t->helix_deg[k]) || !finite(t->tooth_deg[k]) || fabs(t->helix_deg[k]) >= 89.0)
            return fail(FSM_E_INVALID, "helix/tooth angles must be finite, |helix| < 89");
    return FSM_OK;
}

static fsm_status check_process(const fsm_process_desc* p) {
    if (!p) return fail(FSM_E_INVALID, "process descriptor is NULL");
    const double vals[] = {p->fz, p->rpm, p->rot_step_deg, p->phase0_deg, p->ap, p->lead_deg, p->tilt_deg,
                           p->ae, p->pass_x0, p->pass_y0, p->stock_z, p->x0, p->y0, p->pitch, p->wall_y,
                           p->feed_dir_deg};
    for (double v : vals)
        if (!finite(v)) return fail(FSM_E_INVALID, "non-finite process value");
    if (!(p->fz > 0.0)) return fail(FSM_E_INVALID, "fz must be > 0");
    if (!(p->ap > 0.0)) return fail(FSM_E_INVALID, "ap must be > 0");
    if (!(p->pitch > 0.0)) return fail(FSM_E_INVALID, "pitch must be > 0");
    if (steps_per_rev(p->rot_step_deg) < 0) return fail(FSM_E_INVALID, "360/rot_step_deg must be an integer");
    if (p->rot_sense != 1 && p->rot_sense != -1) return fail(FSM_E_INVALID, "rot_sense must be +1 or -1");
    if (p->n_passes < 1) return fail(FSM_E_INVALID, "n_passes must be >= 1");
    if (p->steps_per_pass < 1) return fail(FSM_E_INVALID, "steps_per_pass must be >= 1");
    if ((double)p->n_passes * (double)p->steps_per_pass >= 2147483647.0)
        return fail(FSM_E_INVALID, "n_passes * steps_per_pass must be < 2^31");
    if (p->nx < 1 || p->ny < 1 || p->nx > 65535 * 256 || p->ny > 65535 * 256)
        return fail(FSM_E_INVALID, "grid size out of range");
    if ((double)p->nx * (double)p->ny > 4.0e9) return fail(FSM_E_INVALID, "grid larger than 4e9 cells");
    if (fabs(p->lead_deg) >= 89.0 || fabs(p->tilt_deg) >= 89.0) return fail(FSM_E_INVALID, "|lead|, |tilt| < 89");
    if (p->precision != FSM_FP64 && p->precision != FSM_FP32) return fail(FSM_E_INVALID, "unknown precision");
    if (p->surface != FSM_SURFACE_FLOOR && p->surface != FSM_SURFACE_WALL)
        return fail(FSM_E_INVALID, "unknown surface");
    if (p->surface == FSM_SURFACE_WALL && p->n_passes != 1)
        return fail(FSM_E_INVALID, "a wall map takes a single pass");
    if (p->pass_mode != FSM_PASS_ONE_WAY && p->pass_mode != FSM_PASS_ZIGZAG)
        return fail(FSM_E_INVALID, "unknown pass_mode");
    if (p->surface == FSM_SURFACE_WALL && feed_tilted(*p))
        return fail(FSM_E_INVALID, "a wall map takes the +X feed (feed_dir_deg a multiple of 360)");
    return FSM_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Tile width for a surface whose feed per revolution spans rev cells: a
// whole number k of revolutions, less the visits' margins (two cells each
// side), so that every spindle phase brings a point over the tile on the
// same number k of revolutions -- the phase form's visit count is then the
// same on nearly every lane. k is near target / rev, the targets measured
// on GB300: 700 cells for FP32 maps (8 mm flat floor 704x55 17.0 ms vs
// 468x83 17.9 ms, side wall 704x55 0.60 ms vs 0.63 ms; the ball raster's
// 320-cell revolutions give 636 either way), 1280 for FP64 floors, whose
// phase form computes the FP64 height once per phase and gains from more
// revolutions per tile (ball raster 1276x17 1.91 ms vs 636x34 2.09 ms; flat
// floor 1296x16 28.6 ms vs 468x46 28.9 ms), 480 for FP64 walls (468x46
// 1.52 ms vs 940x23 2.36 ms). 0 when the feed per revolution is too long
// for the widths allowed (64 .. 1.5 target).
static int feed_aligned_width(const fsm_process_desc& p, int n_teeth) {
    const double target = p.precision == FSM_FP32 ? 700.0 : (p.surface == FSM_SURFACE_FLOOR ? 1280.0 : 480.0);
    const double rev = (double)n_teeth * p.fz / p.pitch;
    if (!(rev > 0.0) || rev > 1.5 * target) return 0;
    const int k = std::max(1, (int)llround(target / rev));
    const int w = ((int)floor((double)k * rev) - 4) & ~3;
    return (w >= 64 && w <= (int)(1.5 * target)) ? w : 0;
}

Shape pick_shape(const fsm_process_desc& p, const fsm_predict_opts* o, const fsm_process_desc* const* group,
                 int n_group, int sm_count, const fsm_tool_desc* const* tools) {
    // Default ladder, measured on GB300: 16 warps sharing one large, wide
    // tile amortise the per-tile work best, and the tile takes all the
    // shared memory the 16 warps' scratch leaves: 512x76 FP32 cells
    // (152 KB) and 640x34 FP64 cells (170 KB). Measured on the 5x5 mm, 1 um
    // ball raster in feed-aligned widths: FP32 636x61 0.985 ms vs 636x45
    // 1.06 ms, 636x36 1.18 ms; FP64 632x34 2.09 ms vs 632x27 2.32 ms; more
    // warps on smaller tiles were slower (20 warps, 636x36: 1.31 ms), fewer
    // warps on larger ones too (12 warps, 636x57: 1.12 ms). Wide, short
    // tiles keep per-arc x ranges tight. A step down to 8-warp CTAs, two
    // per SM, is taken while the surfaces have fewer tiles than there are
    // resident CTAs by more than half (small maps: the 2 Mcell face-milled
    // patch runs 0.33 ms at 128x32 against 0.99 ms at 512x48; the 20x1 mm
    // wall's 140 tiles of 468x83 fill 152 SMs well: 0.63 ms against 6.3 ms
    // at 256x48).
    struct Level { int tx, ty, threads, ctas; };
    static const Level l32[] = {{512, 76, 512, 1}, {256, 48, 256, 2}, {128, 32, 256, 2}};
    static const Level l64[] = {{640, 34, 512, 1}, {256, 32, 256, 2}, {128, 32, 256, 2}};
    const Level* lv = p.precision == FSM_FP64 ? l64 : l32;
    int pick = 0;
    if (group && n_group > 0 && sm_count > 0) {
        for (pick = 0; pick < 2; ++pick) {
            long long tiles = 0;
            for (int i = 0; i < n_group; ++i)
                if (group[i]->precision == p.precision)
                    tiles += (long long)((group[i]->nx + lv[pick].tx - 1) / lv[pick].tx) *
                             ((group[i]->ny + lv[pick].ty - 1) / lv[pick].ty);
            if (2 * tiles >= (long long)sm_count * lv[pick].ctas) break;
        }
    }
    Shape s;
    s.tile_x = lv[pick].tx;
    s.tile_y = lv[pick].ty;
    s.threads = lv[pick].threads;
    // a lone surface of this precision on the large tiles: the same cell
    // budget in a width aligned to its feed per revolution (measured: 8 mm
    // flat-end floor 21.7 -> 20.7 ms, side wall 1.03 -> 0.91 ms, FP64 ball
    // raster 2.54 -> 2.52 ms)
    if (pick == 0 && group && tools && n_group > 0) {
        int lone = -1, count = 0;
        for (int i = 0; i < n_group; ++i)
            if (group[i]->precision == p.precision) {
                lone = i;
                ++count;
            }
        const int w = count == 1 ? feed_aligned_width(*group[lone], tools[lone]->n_teeth) : 0;
        if (w > 0) {
            s.tile_y = std::max(1, s.tile_x * s.tile_y / w);
            s.tile_x = w;
        }
    }
    // surfaces fed off the X axis: the tile of the same cell budget whose
    // extent along (A) and across (B) the feed minimises B (A + 160) / cells,
    // aspect at most 10: the phases enumerated grow with B, each run's
    // steps with A plus a slack of about 160 cells (fitted to the 5 mm ball
    // raster at 10, 30 and 90 degrees: 90 degrees runs 56x512 in 1.72 ms
    // against 2.03 ms square, 30 degrees is fastest near square). Surfaces
    // fed in different directions take a square tile.
    if (group && n_group > 0) {
        bool all_tilted = false, same_dir = true, first = true;
        double dir = 0.0;
        for (int i = 0; i < n_group; ++i)
            if (group[i]->precision == p.precision) {
                all_tilted = feed_tilted(*group[i]);
                if (!all_tilted) break;
                const double d = fmod(fmod(group[i]->feed_dir_deg, 180.0) + 180.0, 180.0);
                if (!first && d != dir) same_dir = false;
                dir = d;
                first = false;
            }
        if (all_tilted) {
            const int cells = s.tile_x * s.tile_y;
            const int side = std::max(4, (int)floor(sqrt((double)cells)) & ~3);
            s.tile_x = side;
            s.tile_y = std::max(1, cells / side);
            if (same_dir) {
                const double c = fabs(cos(dir * (M_PI / 180.0))), sn = fabs(sin(dir * (M_PI / 180.0)));
                double best = 1e300;
                for (int tx = 16; tx <= 1024; tx += 4) {
                    const int ty = cells / tx;
                    if (ty < 8 || tx > 10 * ty || ty > 10 * tx) continue;
                    const double A = tx * c + ty * sn, B = tx * sn + ty * c;
                    const double cost = B * (A + 160.0) / ((double)tx * ty);
                    if (cost < best) {
                        best = cost;
                        s.tile_x = tx;
                        s.tile_y = ty;
                    }
                }
            }
        }
    }
    if (o) {
        if (o->tile_x > 0) s.tile_x = o->tile_x;
        if (o->tile_y > 0) s.tile_y = o->tile_y;
        if (o->block_threads > 0) s.threads = o->block_threads;
    }
    return s;
}

// Copy the descriptors into a device plan; table pointers relative to base.
size_t fill_surface(const fsm_tool_desc& t, const fsm_process_desc& p, const Shape& sh, Surface* s,
                    char* base) {
    memset(s, 0, sizeof *s);
    s->kind = t.kind;
    s->n_teeth = t.n_teeth;
    s->n_edge = t.n_edge;
    s->n_end = (t.kind == FSM_TOOL_FLAT || t.kind == FSM_TOOL_TORUS) ? t.n_end : 0;
    s->corner_radius = t.corner_radius;
    s->diameter = t.diameter;
    s->runout_mm = t.runout_mm;
    s->runout_phase_deg = t.runout_phase_deg;
    for (int k = 0; k < FSM_MAX_TEETH; ++k) {
        s->helix_deg[k] = t.kind == FSM_TOOL_INSERT ? 0.0 : t.helix_deg[k];
        s->tooth_deg[k] = t.tooth_deg[k];
    }
    s->insert_radius = t.insert_radius;
    s->rake_f_deg = t.rake_f_deg;
    s->rake_p_deg = t.rake_p_deg;
    s->eps_r_mm = t.eps_r_mm;
    s->eps_a_mm = t.eps_a_mm;
    s->fz = p.fz;
    s->rot_step_deg = p.rot_step_deg;
    s->phase0_deg = p.phase0_deg;
    s->rot_sense = p.rot_sense;
    s->n_passes = p.n_passes;
    s->ap = p.ap;
    s->lead_deg = p.lead_deg;
    s->tilt_deg = p.tilt_deg;
    s->ae = p.ae;
    s->pass_x0 = p.pass_x0;
    s->pass_y0 = p.pass_y0;
    s->steps_per_pass = (int32_t)p.steps_per_pass;
    s->S = (int32_t)steps_per_rev(p.rot_step_deg);
    s->stock_z = p.stock_z;
    s->surface = p.surface;
    s->wall_y = p.wall_y;
    s->pass_mode = p.pass_mode;
    s->feed_dir_deg = p.feed_dir_deg;
    s->tilted = feed_tilted(p) ? 1 : 0;
    s->x0 = p.x0;
    s->y0 = p.y0;
    s->pitch = p.pitch;
    s->nx = p.nx;
    s->ny = p.ny;
    s->precision = p.precision;
    s->E = s->n_edge + s->n_end;
    s->tile_x = sh.tile_x;
    s->tile_y = sh.tile_y;
    s->ntx = (p.nx + sh.tile_x - 1) / sh.tile_x;
    s->nty = (p.ny + sh.tile_y - 1) / sh.tile_y;
    const size_t NE = (size_t)s->n_teeth * (size_t)s->E;
    const size_t G = (size_t)s->n_teeth * (size_t)((s->E + 31) / 32);
    size_t off = 0;
    s->tool32 = (float4*)(base + off);
    off += align256(NE * 4 * sizeof(float4));
    s->tool64 = (double*)(base + off);
    off += align256(NE * 9 * sizeof(double));
    s->ph32 = (float2*)(base + off);
    off += align256(2 * (size_t)s->S * sizeof(float2));
    s->ph64 = (double2*)(base + off);
    off += align256(2 * (size_t)s->S * sizeof(double2));
    s->groups = (float4*)(base + off);
    off += align256(G * sizeof(float4));
    s->plan_part = (double*)(base + off);
    off += align256(sizeof(double) * 4 * kPlanParts);
    s->tile_queue = (int*)(base + off);
    off += 256;
    return off;
}

size_t surface_table_bytes(const fsm_tool_desc& t, const fsm_process_desc& p) {
    Surface s;
    return fill_surface(t, p, pick_shape(p, nullptr), &s, nullptr);
}

size_t surface_overhead_bytes(const fsm_tool_desc& t, const fsm_process_desc& p) {
    Surface s;
    const Shape sh = pick_shape(p, nullptr);
    return align256(sizeof(Surface)) + fill_surface(t, p, sh, &s, nullptr) + 64 * 1024;
}

}  // namespace fsm

using namespace fsm;

extern "C" {

const char* fsm_last_error(fsm_ctx*) { return g_err.c_str(); }

fsm_status fsm_create_context(int device, fsm_ctx** out) {
    if (!out) return fail(FSM_E_INVALID, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(FSM_E_INVALID, "no such CUDA device");
    DeviceGuard dev_guard(device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor < 100)
        return fail(FSM_E_CUDA, "the library is built for sm_103a (Blackwell Ultra)");
    // make sure our kernels are loadable on this device and may use all of
    // its opt-in shared memory
    if ((e = fsm::sweep_allow_smem(prop.sharedMemPerBlockOptin)) != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "kernel image not loadable on this device");
    }
    size_t smem = fsm::sweep_smem_bytes(FSM_FP32, 8, 8, 256);
    if (fsm::sweep_blocks_per_sm(FSM_FP32, 256, smem) <= 0) {
        cudaGetLastError();
        return fail(FSM_E_CUDA, "kernel image not loadable on this device");
    }
    fsm_ctx* c = new fsm_ctx();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *out = c;
    return FSM_OK;
}

fsm_status fsm_destroy_context(fsm_ctx* ctx) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    if (ctx->server) fsm_server_stop(ctx);
    delete ctx;
    return FSM_OK;
}

fsm_status fsm_create_tool(fsm_ctx* ctx, const fsm_tool_desc* desc, fsm_tool** out) {
    if (!ctx || !out) return fail(FSM_E_INVALID, "ctx/out is NULL");
    fsm_status st = check_tool(desc);
    if (st != FSM_OK) return st;
    fsm_tool* t = new fsm_tool();
    t->d = *desc;
    *out = t;
    return FSM_OK;
}

fsm_status fsm_destroy_tool(fsm_ctx*, fsm_tool* tool) {
    delete tool;
    return FSM_OK;
}

fsm_status fsm_set_process(fsm_ctx* ctx, const fsm_process_desc* desc, fsm_process** out) {
    if (!ctx || !out) return fail(FSM_E_INVALID, "ctx/out is NULL");
    fsm_status st = check_process(desc);
    if (st != FSM_OK) return st;
    fsm_process* p = new fsm_process();
    p->d = *desc;
    *out = p;
    return FSM_OK;
}

fsm_status fsm_destroy_process(fsm_ctx*, fsm_process* proc) {
    delete proc;
    return FSM_OK;
}

}  // extern "C"

namespace fsm {

// Launch configuration of the sweep for one precision; checks shared memory.
fsm_status sweep_config(fsm_ctx* ctx, int precision, const Shape& sh, size_t* smem, int* blocks_per_sm) {
    if (sh.threads < 64 || sh.threads > 512 || (sh.threads & 31))
        return fail(FSM_E_INVALID, "block_threads must be a multiple of 32 in 64..512");
    if (sh.tile_x < 4 || sh.tile_y < 1 || (sh.tile_x & 3)) return fail(FSM_E_INVALID, "tile_x must be a multiple of 4");
    *smem = sweep_smem_bytes(precision, sh.tile_x, sh.tile_y, sh.threads);
    if (*smem + sweep_static_bytes() > ctx->smem_optin) return fail(FSM_E_INVALID, "tile does not fit in shared memory");
    // the occupancy queries cost host time on every call: cached per context
    const std::array<long long, 3> key = {precision, sh.threads, (long long)*smem};
    int b = -1;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->occupancy.find(key);
        if (it != ctx->occupancy.end()) b = it->second;
    }
    if (b < 0) {
        b = sweep_blocks_per_sm(precision, sh.threads, *smem);
        if (b > 0) {
            std::lock_guard<std::mutex> lk(ctx->mu);
            ctx->occupancy[key] = b;
        }
    }
    if (b <= 0) {
        cudaGetLastError();
        return fail(FSM_E_CUDA, "sweep kernel cannot be resident with this configuration");
    }
    *blocks_per_sm = b;
    return FSM_OK;
}

std::string tune_key(const fsm_tool_desc& t, const fsm_process_desc& p) {
    char buf[256];
    snprintf(buf, sizeof buf, "%d/%d/%d/%d/%d/%d/%.6g/%d/%d/%.6g/%d", p.surface, p.precision, t.kind, t.n_teeth,
             t.n_edge + ((t.kind == FSM_TOOL_FLAT || t.kind == FSM_TOOL_TORUS) ? t.n_end : 0),
             (int)steps_per_rev(p.rot_step_deg), t.diameter,
             p.nx, p.ny, p.pitch, feed_tilted(p) ? 1 : 0);
    return buf;
}

// FP32 maps decide a point's cell from FP32 tile-local coordinates unless it
// lies within a guard band (the FP32 error bound, in cells) of a boundary;
// the check of an ambiguous point looks one cell to each side, so the band
// must stay below half a cell. This bounds the band of every run of the
// workload from the tool's size, the tile and the whole pass length (the
// device takes each run's own, smaller, figures) and rejects FP32 maps whose
// pitch is too fine for it -- about 20 nm and below for a 10 mm tool -- for
// which FP64 maps are the choice.
fsm_status check_fp32_band(const fsm_tool_desc& t, const fsm_process_desc& p, const Shape& sh) {
    if (p.precision != FSM_FP32) return FSM_OK;
    const double u24 = 5.9604644775390625e-8;
    const double r_max = 0.5 * t.diameter + t.insert_radius +
                         (double)t.n_teeth * (fabs(t.eps_r_mm) + fabs(t.eps_a_mm)) + t.runout_mm;
    const double w_sum = 3.0 * (t.diameter + p.ap + t.insert_radius + (double)t.n_teeth * fabs(t.eps_a_mm));
    const double tile = (double)std::max(sh.tile_x, sh.tile_y);
    const double span = (double)p.steps_per_pass * (double)t.n_teeth * p.fz * p.rot_step_deg / 360.0;
    const double band = 1.5 * u24 * (6.0 * r_max + 3.0 * w_sum + 3.0 * tile * p.pitch + 2.0 * span) / p.pitch +
                        3.0 * u24 * tile + 1e-6;
    if (band >= 0.45)
        return fail(FSM_E_INVALID, "pitch too fine for an FP32 map of this tool and pass (FP32 guard band of " +
                                       std::to_string(band) + " cells); use FSM_FP64");
    return FSM_OK;
}

fsm_status check_opts(const fsm_predict_opts* o, const fsm_process_desc* const*, int) {
    if (o && o->sweep_form != FSM_FORM_AUTO && o->sweep_form != FSM_FORM_ITEM && o->sweep_form != FSM_FORM_PHASE)
        return fail(FSM_E_INVALID, "sweep_form must be FSM_FORM_AUTO, FSM_FORM_ITEM or FSM_FORM_PHASE");
    return FSM_OK;
}

fsm_status predict_one(fsm_ctx* ctx, const fsm_tool_desc& t, const fsm_process_desc& p, void* d_heights,
                       const fsm_predict_opts* opts, cudaStream_t st) {
    const fsm_process_desc* self = &p;
    if (fsm_status rc0 = check_opts(opts, &self, 1)) return rc0;
    const fsm_tool_desc* self_tool = &t;
    Shape sh = pick_shape(p, opts, &self, 1, ctx->sm_count, &self_tool);
    fsm_predict_opts tuned_opts;
    if (!opts || opts->tile_x <= 0) {  // an autotuned shape for this workload, if any
        std::lock_guard<std::mutex> lk(ctx->mu);
        auto it = ctx->tuned.find(tune_key(t, p));
        if (it != ctx->tuned.end()) {
            sh.tile_x = it->second[0];
            sh.tile_y = it->second[1];
            sh.threads = it->second[3];
            if (opts) tuned_opts = *opts;
            else memset(&tuned_opts, 0, sizeof tuned_opts);
            tuned_opts.ctas_per_sm = it->second[2];
            opts = &tuned_opts;
        }
    }
    size_t smem = 0;
    int bps = 0;
    fsm_status rc = check_fp32_band(t, p, sh);
    if (rc != FSM_OK) return rc;
    rc = sweep_config(ctx, p.precision, sh, &smem, &bps);
    if (rc != FSM_OK) return rc;
    Surface s;
    const size_t surf_bytes = align256(sizeof(Surface));
    size_t table_bytes = fill_surface(t, p, sh, &s, nullptr);
    void* ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, surf_bytes + table_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (tables)");
    fill_surface(t, p, sh, &s, (char*)ws + surf_bytes);
    s.heights = d_heights;
    s.form = opts ? opts->sweep_form : FSM_FORM_AUTO;
    s.form_tasks = opts ? (unsigned long long*)opts->d_form_tasks : nullptr;
    Surface* d_s = (Surface*)ws;
    if ((e = launch_plan(d_s, 1, &s, 0, ctx->sm_count, st)) != cudaSuccess) {
        cudaFreeAsync(ws, st);
        return cuda_fail(e, "plan kernel");
    }
    const int tiles = s.ntx * s.nty;
    if (opts && opts->ctas_per_sm > 0) bps = std::min(bps, (int)opts->ctas_per_sm);
    const int grid = std::min(tiles, ctx->sm_count * bps);
    if (opts && opts->sweep_events[0]) cudaEventRecord((cudaEvent_t)opts->sweep_events[0], st);
    // tiles are handed out by a device counter that the planning kernel zeroed
    e = launch_sweep_shaped(p.precision, d_s, 1, nullptr, tiles, s.tile_queue,
                            opts ? (long long*)opts->d_counters : nullptr, grid, sh.threads, smem, st,
                            phase_form_pays(t, p, sh.tile_x, s.form), feed_tilted(p));
    if (opts && opts->sweep_events[1]) cudaEventRecord((cudaEvent_t)opts->sweep_events[1], st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep kernel");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return FSM_OK;
}

fsm_status trajectory_one(fsm_ctx* ctx, const fsm_tool_desc& t, const fsm_process_desc& p, fsm_traj_point* d_out,
                          int64_t capacity, cudaStream_t st) {
    const long long n_rec = (long long)p.n_passes * p.steps_per_pass * t.n_teeth;
    if (capacity < n_rec) return fail(FSM_E_INVALID, "trajectory buffer holds fewer records than the tool path");
    if (((uintptr_t)d_out & 15) != 0) return fail(FSM_E_INVALID, "d_out must be 16-byte aligned");
    Shape sh = pick_shape(p, nullptr);
    Surface s;
    const size_t surf_bytes = align256(sizeof(Surface));
    const size_t table_bytes = fill_surface(t, p, sh, &s, nullptr);
    const size_t jmin_bytes = align256((size_t)s.S * (size_t)t.n_teeth * sizeof(int32_t));
    void* ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, surf_bytes + table_bytes + jmin_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (trajectory tables)");
    fill_surface(t, p, sh, &s, (char*)ws + surf_bytes);
    s.heights = nullptr;
    Surface* d_s = (Surface*)ws;
    if ((e = launch_plan(d_s, 1, &s, 0, ctx->sm_count, st)) == cudaSuccess)
        e = launch_trajectory(d_s, s.S, t.n_teeth, n_rec, (int32_t*)((char*)ws + surf_bytes + table_bytes), d_out,
                              st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "trajectory kernels");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return FSM_OK;
}

fsm_status roughness_one(fsm_ctx*, const void* d_h, int precision, int nx, int ny, int n_rows, int n_cols,
                         fsm_roughness_out* d_out, cudaStream_t st) {
    RoughJob jb;
    jb.h = d_h;
    jb.n = (size_t)nx * (size_t)ny;
    jb.nx = nx;
    jb.ny = ny;
    jb.n_rows = n_rows;
    jb.n_cols = n_cols;
    jb.out = d_out;
    char* ws = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&ws, roughness_one_ws_bytes(jb.n), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (roughness)");
    e = launch_roughness_one(precision, jb, ws, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "roughness kernels");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return FSM_OK;
}

}  // namespace fsm

extern "C" {

fsm_status fsm_predict_surface(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc, void* d_heights,
                               const fsm_predict_opts* opts, void* stream) {
    if (!ctx || !tool || !proc) return fail(FSM_E_INVALID, "ctx/tool/proc is NULL");
    if (!d_heights) return fail(FSM_E_INVALID, "d_heights is NULL");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    return fsm::predict_one(ctx, tool->d, proc->d, d_heights, opts, (cudaStream_t)stream);
}

fsm_status fsm_trajectory_records(const fsm_tool* tool, const fsm_process* proc, int64_t* n) {
    if (!tool || !proc || !n) return fail(FSM_E_INVALID, "tool/proc/n is NULL");
    *n = (int64_t)proc->d.n_passes * proc->d.steps_per_pass * tool->d.n_teeth;
    return FSM_OK;
}

fsm_status fsm_predict_trajectory(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc,
                                  fsm_traj_point* d_out, int64_t capacity, void* stream) {
    if (!ctx || !tool || !proc) return fail(FSM_E_INVALID, "ctx/tool/proc is NULL");
    if (!d_out) return fail(FSM_E_INVALID, "d_out is NULL");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    return fsm::trajectory_one(ctx, tool->d, proc->d, d_out, capacity, (cudaStream_t)stream);
}

fsm_status fsm_roughness(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx, int32_t ny,
                         int32_t n_rows, int32_t n_cols, fsm_roughness_out* d_out, void* stream) {
    if (!ctx || !d_heights || !d_out) return fail(FSM_E_INVALID, "ctx/d_heights/d_out is NULL");
    if (precision != FSM_FP64 && precision != FSM_FP32) return fail(FSM_E_INVALID, "unknown precision");
    if (nx < 1 || ny < 1) return fail(FSM_E_INVALID, "nx, ny must be >= 1");
    if (n_rows < 0 || n_cols < 0 || n_rows > FSM_MAX_PROFILES || n_cols > FSM_MAX_PROFILES)
        return fail(FSM_E_INVALID, "0 <= n_rows, n_cols <= 16");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    return fsm::roughness_one(ctx, d_heights, precision, nx, ny, n_rows, n_cols, d_out, (cudaStream_t)stream);
}

fsm_status fsm_moment_partials(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx, int32_t ny,
                               double about, double* d_out, void* stream) {
    if (!ctx || !d_heights || !d_out) return fail(FSM_E_INVALID, "ctx/d_heights/d_out is NULL");
    if (precision != FSM_FP64 && precision != FSM_FP32) return fail(FSM_E_INVALID, "unknown precision");
    if (nx < 1 || ny < 1) return fail(FSM_E_INVALID, "nx, ny must be >= 1");
    if (!isfinite(about)) return fail(FSM_E_INVALID, "about must be finite");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    const size_t n = (size_t)nx * (size_t)ny;
    cudaStream_t st = (cudaStream_t)stream;
    double* ws = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&ws, moment_ws_bytes(n), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync (moments)");
    e = launch_moments(precision, d_heights, n, about, ws, d_out, st);
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "moment kernels");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return FSM_OK;
}

}  // extern "C"

extern "C" fsm_status fsm_autotune(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc, void* d_heights,
                                   int32_t max_candidates, fsm_predict_opts* best, float* best_ms, void* stream) {
    if (!ctx || !tool || !proc || !d_heights || !best) return fail(FSM_E_INVALID, "NULL argument");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    cudaStream_t st = (cudaStream_t)stream;
    // candidates (tile_x, tile_y, threads): wide, short tiles shared by many
    // warps first (they amortise the enumeration and keep x ranges tight)
    static const int c32[][3] = {{512, 76, 512}, {640, 60, 512}, {768, 50, 512}, {1024, 38, 512}, {384, 100, 512},
                                 {512, 56, 512}, {256, 150, 512}, {512, 24, 256}, {256, 48, 256}, {256, 64, 256},
                                 {128, 48, 256}, {128, 32, 256}, {64, 32, 256}};
    static const int c64[][3] = {{640, 34, 512}, {512, 42, 512}, {768, 28, 512}, {256, 84, 512}, {512, 24, 384},
                                 {256, 32, 256}, {128, 64, 256}, {128, 32, 256}, {64, 64, 256}, {64, 32, 256}};
    const bool f64 = proc->d.precision == FSM_FP64;
    const int nlist = f64 ? 10 : 13;
    // the default shape (feed-aligned where it applies) is tried first
    const fsm_process_desc* self = &proc->d;
    const fsm_tool_desc* self_tool = &tool->d;
    const Shape def = pick_shape(proc->d, nullptr, &self, 1, ctx->sm_count, &self_tool);
    const int nshape = nlist + 1;
    auto cand = [&](int si, int k) -> int {
        if (si == 0) return k == 0 ? def.tile_x : k == 1 ? def.tile_y : def.threads;
        return f64 ? c64[si - 1][k] : c32[si - 1][k];
    };
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    float best_t = 1e30f;
    fsm_predict_opts bo;
    memset(&bo, 0, sizeof bo);
    int tried = 0;
    fsm_status rc = FSM_OK;
    for (int si = 0; si < nshape && rc == FSM_OK; ++si) {
        for (int cps = 2; cps >= 1 && rc == FSM_OK; --cps) {
            if (max_candidates > 0 && tried >= max_candidates) break;
            fsm_predict_opts o;
            memset(&o, 0, sizeof o);
            o.tile_x = cand(si, 0);
            o.tile_y = cand(si, 1);
            o.block_threads = cand(si, 2);
            o.ctas_per_sm = cps;
            size_t smem;
            int bps;
            Shape sh{o.tile_x, o.tile_y, o.block_threads};
            if (sweep_config(ctx, proc->d.precision, sh, &smem, &bps) != FSM_OK) continue;
            if (bps < cps) continue;
            ++tried;
            // one warm run, then one timed run
            rc = predict_one(ctx, tool->d, proc->d, d_heights, &o, st);
            if (rc != FSM_OK) break;
            o.sweep_events[0] = ev[0];
            o.sweep_events[1] = ev[1];
            rc = predict_one(ctx, tool->d, proc->d, d_heights, &o, st);
            if (rc != FSM_OK) break;
            if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rc = cuda_fail(e, "autotune synchronise");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (ms < best_t) {
                best_t = ms;
                bo = o;
                bo.sweep_events[0] = bo.sweep_events[1] = nullptr;
            }
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != FSM_OK) return rc;
    if (tried == 0) return fail(FSM_E_INVALID, "no sweep configuration fits this device");
    *best = bo;
    if (best_ms) *best_ms = best_t;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tuned[tune_key(tool->d, proc->d)] = {bo.tile_x, bo.tile_y, bo.ctas_per_sm, bo.block_threads};
    return FSM_OK;
}
