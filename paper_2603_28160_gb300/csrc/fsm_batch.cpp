// fsm_batch.cpp -- many surfaces in one persistent launch per precision.
//
// A batch lays out, in one device buffer: the per-surface plans (FP64 group
// first, then FP32), the tile prefix of each group, two work-queue counters,
// the roughness jobs and chunk prefixes, the roughness scratch and every
// surface's tables. Running it enqueues: a memset of the queues, the plan
// kernel (one block per surface), one persistent sweep per precision group
// and the chunked roughness launches.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/fsm.h"
#include "fsm_host.h"
#include "fsm_internal.h"

namespace fsm {

struct BatchLayout {
    int n = 0, n64 = 0, n32 = 0;
    int tiles64 = 0, tiles32 = 0;
    int chunks64 = 0, chunks32 = 0;
    int max_prof = 0;
    Shape sh64{}, sh32{};
    size_t smem64 = 0, smem32 = 0;
    int bps64 = 0, bps32 = 0;
    size_t off_surf = 0, off_tb64 = 0, off_tb32 = 0, off_queue = 0, off_jobs = 0, off_cb64 = 0,
           off_cb32 = 0, off_part64 = 0, off_part32 = 0, off_tables = 0, total = 0;
    bool rough = false;
    bool phase_form32 = false, phase_form64 = false;  // some surface's runs come back for many revolutions
    bool tilt32 = false, tilt64 = false;              // some surface is fed off the X axis
    int plan_work = 0;  // largest (edge points + phases) of a surface, for the planning grid
    long long* counters = nullptr;
    void* events[2] = {nullptr, nullptr};
    std::vector<char> blob;  // host image of [off_surf, off_tables)
};

// Build the host image of a batch and its layout. `base` = device address of
// the buffer (NULL to size only).
fsm_status build_batch(fsm_ctx* ctx, int n, const fsm_tool_desc* const* tools,
                       const fsm_process_desc* const* procs, void* const* heights,
                       fsm_roughness_out* d_rough, const fsm_predict_opts* opts, char* base, BatchLayout* L,
                       const TableRef* trefs = nullptr) {
    if (n < 1) return fail(FSM_E_INVALID, "batch size must be >= 1");
    if (fsm_status rc0 = check_opts(opts, procs, n)) return rc0;
    const int form = opts ? opts->sweep_form : FSM_FORM_AUTO;
    std::vector<int> order;
    order.reserve(n);
    for (int grp = 0; grp < 2; ++grp)
        for (int i = 0; i < n; ++i)
            if ((procs[i]->precision == FSM_FP64) == (grp == 0)) order.push_back(i);
    L->n = n;
    L->n64 = 0;
    for (int i = 0; i < n; ++i) L->n64 += procs[i]->precision == FSM_FP64;
    L->n32 = n - L->n64;
    fsm_process_desc p64 = *procs[0], p32 = *procs[0];
    p64.precision = FSM_FP64;
    p32.precision = FSM_FP32;
    L->sh64 = pick_shape(p64, opts, procs, n, ctx->sm_count, tools);
    L->sh32 = pick_shape(p32, opts, procs, n, ctx->sm_count, tools);
    fsm_status rc;
    if (L->n64 && (rc = sweep_config(ctx, FSM_FP64, L->sh64, &L->smem64, &L->bps64)) != FSM_OK) return rc;
    if (L->n32 && (rc = sweep_config(ctx, FSM_FP32, L->sh32, &L->smem32, &L->bps32)) != FSM_OK) return rc;
    L->rough = d_rough != nullptr;
    for (int i = 0; i < n; ++i) {
        const bool f64 = procs[i]->precision == FSM_FP64;
        if (phase_form_pays(*tools[i], *procs[i], f64 ? L->sh64.tile_x : L->sh32.tile_x, form))
            (f64 ? L->phase_form64 : L->phase_form32) = true;
        if (feed_tilted(*procs[i])) (f64 ? L->tilt64 : L->tilt32) = true;
    }
    L->counters = opts ? (long long*)opts->d_counters : nullptr;
    if (opts) {
        L->events[0] = opts->sweep_events[0];
        L->events[1] = opts->sweep_events[1];
        if (opts->ctas_per_sm > 0) {
            L->bps64 = std::min(L->bps64, (int)opts->ctas_per_sm);
            L->bps32 = std::min(L->bps32, (int)opts->ctas_per_sm);
        }
    }

    // sizes
    std::vector<Surface> hs(n);
    std::vector<size_t> toff(n);
    size_t tables = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const Shape& sh = procs[i]->precision == FSM_FP64 ? L->sh64 : L->sh32;
        if ((rc = check_fp32_band(*tools[i], *procs[i], sh)) != FSM_OK) return rc;
        toff[k] = tables;
        const size_t tb = fill_surface(*tools[i], *procs[i], sh, &hs[k], nullptr);
        if (!trefs || !trefs[i].base) tables += tb;  // tables held elsewhere take no batch space
        L->plan_work = std::max(L->plan_work, hs[k].n_teeth * hs[k].E + hs[k].S);
    }
    std::vector<int> tb64(L->n64 + 1, 0), tb32(L->n32 + 1, 0), cb64(L->n64 + 1, 0), cb32(L->n32 + 1, 0);
    for (int k = 0; k < n; ++k) {
        const size_t cells = (size_t)hs[k].nx * (size_t)hs[k].ny;
        const int tiles = hs[k].ntx * hs[k].nty;
        const int chunks = (int)((cells + kChunk - 1) / kChunk);
        if (k < L->n64) {
            tb64[k + 1] = tb64[k] + tiles;
            cb64[k + 1] = cb64[k] + chunks;
        } else {
            tb32[k - L->n64 + 1] = tb32[k - L->n64] + tiles;
            cb32[k - L->n64 + 1] = cb32[k - L->n64] + chunks;
        }
    }
    L->tiles64 = tb64[L->n64];
    L->tiles32 = tb32[L->n32];
    L->chunks64 = cb64[L->n64];
    L->chunks32 = cb32[L->n32];
    L->max_prof = 20;
    size_t off = 0;
    L->off_surf = off;  off += align256(sizeof(Surface) * n);
    L->off_tb64 = off;  off += align256(sizeof(int) * (L->n64 + 1));
    L->off_tb32 = off;  off += align256(sizeof(int) * (L->n32 + 1));
    L->off_queue = off; off += 256;
    L->off_jobs = off;  off += align256(sizeof(RoughJob) * n);
    L->off_cb64 = off;  off += align256(sizeof(int) * (L->n64 + 1));
    L->off_cb32 = off;  off += align256(sizeof(int) * (L->n32 + 1));
    const size_t blob_end = off;
    // per group: 7 partial sums per chunk, then the sync words of its maps
    L->off_part64 = off;
    off += align256(sizeof(double) * rough_part_doubles(L->chunks64, L->n64, L->max_prof) + rough_sync_bytes(L->n64));
    L->off_part32 = off;
    off += align256(sizeof(double) * rough_part_doubles(L->chunks32, L->n32, L->max_prof) + rough_sync_bytes(L->n32));
    L->off_tables = off; off += tables;
    L->total = off;
    if (!base) return FSM_OK;

    // host image with device addresses
    L->blob.assign(blob_end, 0);
    char* b = L->blob.data();
    std::vector<RoughJob> jobs(n);
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        const Shape& sh = procs[i]->precision == FSM_FP64 ? L->sh64 : L->sh32;
        const bool held = trefs && trefs[i].base;
        fill_surface(*tools[i], *procs[i], sh, &hs[k], held ? trefs[i].base : base + L->off_tables + toff[k]);
        if (held) {
            hs[k].cached = trefs[i].ready ? 1 : 0;
            hs[k].tile_queue = nullptr;  // the batch's own queue hands out tiles
        }
        hs[k].heights = heights[i];
        hs[k].form = form;
        hs[k].form_tasks = opts ? (unsigned long long*)opts->d_form_tasks : nullptr;
        RoughJob& jb = jobs[k];
        jb.h = heights[i];
        jb.nx = hs[k].nx;
        jb.ny = hs[k].ny;
        jb.n = (size_t)jb.nx * (size_t)jb.ny;
        jb.n_rows = 10;
        jb.n_cols = 10;
        jb.out = d_rough ? d_rough + i : nullptr;
    }
    memcpy(b + L->off_surf, hs.data(), sizeof(Surface) * n);
    memcpy(b + L->off_tb64, tb64.data(), sizeof(int) * tb64.size());
    memcpy(b + L->off_tb32, tb32.data(), sizeof(int) * tb32.size());
    memcpy(b + L->off_jobs, jobs.data(), sizeof(RoughJob) * n);
    memcpy(b + L->off_cb64, cb64.data(), sizeof(int) * cb64.size());
    memcpy(b + L->off_cb32, cb32.data(), sizeof(int) * cb32.size());
    return FSM_OK;
}

fsm_status run_batch(fsm_ctx* ctx, const BatchLayout& L, char* base, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(base + L.off_queue, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (queues)");
    Surface* d_surf = (Surface*)(base + L.off_surf);
    if ((e = launch_plan(d_surf, L.n, nullptr, L.plan_work, ctx->sm_count, st)) != cudaSuccess)
        return cuda_fail(e, "plan kernel");
    int* q = (int*)(base + L.off_queue);
    if (L.events[0]) cudaEventRecord((cudaEvent_t)L.events[0], st);
    if (L.n64) {
        const int grid = std::min(L.tiles64, ctx->sm_count * L.bps64);
        e = launch_sweep_shaped(FSM_FP64, d_surf, L.n64, (const int*)(base + L.off_tb64), L.tiles64, q, L.counters,
                                grid, L.sh64.threads, L.smem64, st, L.phase_form64, L.tilt64);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel (FP64)");
    }
    if (L.n32) {
        const int grid = std::min(L.tiles32, ctx->sm_count * L.bps32);
        e = launch_sweep_shaped(FSM_FP32, d_surf + L.n64, L.n32, (const int*)(base + L.off_tb32), L.tiles32, q + 1,
                                L.counters, grid, L.sh32.threads, L.smem32, st, L.phase_form32, L.tilt32);
        if (e != cudaSuccess) return cuda_fail(e, "sweep kernel (FP32)");
    }
    if (L.events[1]) cudaEventRecord((cudaEvent_t)L.events[1], st);
    if (L.rough) {
        const RoughJob* jobs = (const RoughJob*)(base + L.off_jobs);
        if (L.n64 && (e = launch_roughness_jobs(FSM_FP64, jobs, L.n64, (const int*)(base + L.off_cb64), L.chunks64,
                                                L.max_prof, (double*)(base + L.off_part64),
                                                base + L.off_part64 +
                                                    sizeof(double) * rough_part_doubles(L.chunks64, L.n64, L.max_prof),
                                                st)) != cudaSuccess)
            return cuda_fail(e, "roughness (FP64)");
        if (L.n32 && (e = launch_roughness_jobs(FSM_FP32, jobs + L.n64, L.n32, (const int*)(base + L.off_cb32),
                                                L.chunks32, L.max_prof, (double*)(base + L.off_part32),
                                                base + L.off_part32 +
                                                    sizeof(double) * rough_part_doubles(L.chunks32, L.n32, L.max_prof),
                                                st)) !=
                         cudaSuccess)
            return cuda_fail(e, "roughness (FP32)");
    }
    return FSM_OK;
}

static fsm_status unpack(int n, const fsm_tool* const* tools, const fsm_process* const* procs,
                         void* const* d_heights, std::vector<const fsm_tool_desc*>* td,
                         std::vector<const fsm_process_desc*>* pd) {
    if (n < 1 || !tools || !procs || !d_heights) return fail(FSM_E_INVALID, "bad batch arguments");
    td->resize(n);
    pd->resize(n);
    for (int i = 0; i < n; ++i) {
        if (!tools[i] || !procs[i] || !d_heights[i]) return fail(FSM_E_INVALID, "NULL entry in batch");
        (*td)[i] = &tools[i]->d;
        (*pd)[i] = &procs[i]->d;
    }
    return FSM_OK;
}

// One-shot batch on stream-ordered scratch (used by fsm_predict_batch and the server).
fsm_status predict_batch_descs(fsm_ctx* ctx, int n, const fsm_tool_desc* const* td,
                               const fsm_process_desc* const* pd, void* const* d_heights,
                               fsm_roughness_out* d_rough, const fsm_predict_opts* opts, cudaStream_t st,
                               PinnedSlot* slot, const TableRef* trefs) {
    BatchLayout L;
    fsm_status rc = build_batch(ctx, n, td, pd, d_heights, d_rough, opts, nullptr, &L, trefs);
    if (rc != FSM_OK) return rc;
    char* ws = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&ws, L.total, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(FSM_E_NOMEM, "cudaMallocAsync (batch): out of memory")
                                              : cuda_fail(e, "cudaMallocAsync (batch)");
    }
    rc = build_batch(ctx, n, td, pd, d_heights, d_rough, opts, ws, &L, trefs);
    if (rc == FSM_OK) {
        // stage the image in pinned memory so the copy does not block the host
        if (slot && slot->ensure(L.blob.size()) == cudaSuccess) {
            memcpy(slot->host, L.blob.data(), L.blob.size());
            e = cudaMemcpyAsync(ws, slot->host, L.blob.size(), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaEventRecord(slot->done, st);
        } else {
            e = cudaMemcpyAsync(ws, L.blob.data(), L.blob.size(), cudaMemcpyHostToDevice, st);
        }
        rc = e == cudaSuccess ? run_batch(ctx, L, ws, st) : cuda_fail(e, "cudaMemcpyAsync (batch)");
    }
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (rc == FSM_OK && e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync (batch)");
    return rc;
}

}  // namespace fsm

struct fsm_batch {
    fsm::BatchLayout L;
    char* d_buf = nullptr;
};

using namespace fsm;

extern "C" {

fsm_status fsm_predict_batch(fsm_ctx* ctx, int32_t n, const fsm_tool* const* tools, const fsm_process* const* procs,
                             void* const* d_heights, fsm_roughness_out* d_rough, const fsm_predict_opts* opts,
                             void* stream) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    std::vector<const fsm_tool_desc*> td;
    std::vector<const fsm_process_desc*> pd;
    fsm_status rc = unpack(n, tools, procs, d_heights, &td, &pd);
    if (rc != FSM_OK) return rc;
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    return predict_batch_descs(ctx, n, td.data(), pd.data(), d_heights, d_rough, opts, (cudaStream_t)stream,
                               nullptr);
}

fsm_status fsm_batch_create(fsm_ctx* ctx, int32_t n, const fsm_tool* const* tools, const fsm_process* const* procs,
                            void* const* d_heights, fsm_roughness_out* d_rough, const fsm_predict_opts* opts,
                            fsm_batch** out) {
    if (!ctx || !out) return fail(FSM_E_INVALID, "ctx/out is NULL");
    std::vector<const fsm_tool_desc*> td;
    std::vector<const fsm_process_desc*> pd;
    fsm_status rc = unpack(n, tools, procs, d_heights, &td, &pd);
    if (rc != FSM_OK) return rc;
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    fsm_batch* b = new fsm_batch();
    rc = build_batch(ctx, n, td.data(), pd.data(), d_heights, d_rough, opts, nullptr, &b->L);
    if (rc != FSM_OK) {
        delete b;
        return rc;
    }
    if ((e = cudaMalloc((void**)&b->d_buf, b->L.total)) != cudaSuccess) {
        delete b;
        return fail(FSM_E_NOMEM, std::string("cudaMalloc (batch): ") + cudaGetErrorString(e));
    }
    rc = build_batch(ctx, n, td.data(), pd.data(), d_heights, d_rough, opts, b->d_buf, &b->L);
    if (rc == FSM_OK && (e = cudaMemcpy(b->d_buf, b->L.blob.data(), b->L.blob.size(), cudaMemcpyHostToDevice)) !=
                            cudaSuccess)
        rc = cuda_fail(e, "cudaMemcpy (batch)");
    if (rc != FSM_OK) {
        cudaFree(b->d_buf);
        delete b;
        return rc;
    }
    b->L.blob.clear();
    b->L.blob.shrink_to_fit();
    *out = b;
    return FSM_OK;
}

fsm_status fsm_batch_run(fsm_ctx* ctx, fsm_batch* batch, void* stream) {
    if (!ctx || !batch) return fail(FSM_E_INVALID, "ctx/batch is NULL");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    return run_batch(ctx, batch->L, batch->d_buf, (cudaStream_t)stream);
}

fsm_status fsm_batch_destroy(fsm_ctx* ctx, fsm_batch* batch) {
    if (!ctx || !batch) return fail(FSM_E_INVALID, "ctx/batch is NULL");
    DeviceGuard dev_guard(ctx->device);
    cudaError_t e = cudaFree(batch->d_buf);
    delete batch;
    return e == cudaSuccess ? FSM_OK : cuda_fail(e, "cudaFree (batch)");
}

}  // extern "C"
