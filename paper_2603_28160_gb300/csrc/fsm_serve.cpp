// fsm_serve.cpp -- request server with continuous batching.
//
// Requests are admitted first-in first-out while the device memory they need
// (height map + tables + scratch) fits in the budget. Each of n_streams
// slots runs one batch at a time; whenever a slot is idle the scheduler packs
// every admitted request (up to max_batch) into one batched launch on that
// slot's stream, so batches formed from requests that arrived while others
// were running overlap on the device. Completion is signalled by a host
// callback enqueued after the batch; results stay on the device until
// fsm_release_result returns their memory to the budget.
//
// Device-resident state kept across requests: a cache of planned tool tables
// (edge-point tables, phase tables, group bounds) keyed by every input they
// depend on, so a request whose tool and set-up were planned before skips the
// table build; the stream-ordered memory pool keeps freed maps and scratch
// for re-admission instead of returning them to the driver; finished maps
// stay on the device until released.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fsm.h"
#include "fsm_host.h"
#include "fsm_internal.h"

namespace fsm {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// One cached set of planned tables.
struct TableEntry {
    std::string key;
    char* base = nullptr;
    size_t bytes = 0;
    bool ready = false;  // built by a completed launch
    int in_use = 0;      // launches in flight that read or build it
    uint64_t last_use = 0;
};

struct Request {
    uint64_t id = 0;
    fsm_tool_desc tool{};
    fsm_process_desc proc{};
    size_t map_bytes = 0, extra_bytes = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    void* d_heights = nullptr;
    int status = FSM_PENDING;
    bool admitted = false, cancel = false;
    fsm_roughness_out rough{};
    std::shared_ptr<TableEntry> table;  // cached tables this request uses or builds
    bool builds_table = false;
};

struct Slot {
    int index = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // device interval of the running batch
    PinnedSlot staging;
    fsm_roughness_out* h_rough = nullptr;  // pinned, max_batch entries
    fsm_roughness_out* d_rough = nullptr;  // device, max_batch entries
    std::vector<std::shared_ptr<Request>> reqs;
    bool busy = false;
    std::atomic<bool> done{false};
    std::atomic<double> t_done{0.0};
    struct Server* server = nullptr;
};

constexpr size_t kBatchLog = 4096;

struct Server {
    fsm_ctx* ctx = nullptr;
    size_t budget = 0, used = 0, used_peak = 0;
    int max_batch = 1;
    std::vector<std::unique_ptr<Slot>> slots;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread thr;
    bool stop = false;
    uint64_t next_id = 1;
    cudaEvent_t ev_origin = nullptr;  // device time origin of the batch log
    // table cache (least recently used first), its share of the budget
    std::list<std::shared_ptr<TableEntry>> lru;
    std::unordered_map<std::string, std::shared_ptr<TableEntry>> tables;
    size_t table_cap = 0, table_bytes = 0;
    uint64_t tick = 0;
    // statistics and the batch log
    fsm_server_info info{};
    std::vector<fsm_batch_interval> log;
    size_t log_next = 0;
    // fault injection: device allocations still to be reported as failed
    std::atomic<int> fail_allocs{0};
};

// Inputs of the planned tables (plan_kernel, plan_finish_kernel's group
// bounds): the tool, and the process fields that shape the edge points,
// their orientation (feed direction included) and the phase table. Feed, step-over, path, grid and
// precision do not enter them (except a round insert's edge length, which
// depends on fz, and a wall's stock offset).
static std::string table_key(const fsm_tool_desc& t, const fsm_process_desc& p) {
    std::string k;
    auto put = [&](const void* v, size_t n) { k.append((const char*)v, n); };
    put(&t.kind, sizeof t.kind);
    put(&t.n_teeth, sizeof t.n_teeth);
    put(&t.n_edge, sizeof t.n_edge);
    put(&t.n_end, sizeof t.n_end);
    put(&t.diameter, sizeof t.diameter);
    put(t.helix_deg, sizeof(double) * t.n_teeth);
    put(t.tooth_deg, sizeof(double) * t.n_teeth);
    const double v[] = {t.runout_mm, t.runout_phase_deg, t.insert_radius, t.rake_f_deg, t.rake_p_deg, t.eps_r_mm,
                        t.eps_a_mm, t.corner_radius, p.ap, p.lead_deg, p.tilt_deg, p.rot_step_deg, p.phase0_deg,
                        t.kind == FSM_TOOL_INSERT ? p.fz : 0.0,
                        p.surface == FSM_SURFACE_WALL ? p.wall_y - p.pass_y0 : 0.0,
                        feed_tilted(p) ? fmod(p.feed_dir_deg, 360.0) : 0.0};
    put(v, sizeof v);
    put(&p.rot_sense, sizeof p.rot_sense);
    put(&p.surface, sizeof p.surface);
    return k;
}

static void CUDART_CB on_batch_done(void* arg) {
    Slot* s = (Slot*)arg;
    s->t_done.store(now_s());
    s->done.store(true);
    s->server->cv_sched.notify_all();
}

// Reserve cache space for a new entry (server lock held): evict idle
// entries, least recently used first. Returns false if it does not fit.
static bool table_make_room(Server* sv, size_t bytes, cudaStream_t st) {
    if (bytes > sv->table_cap) return false;
    for (auto it = sv->lru.begin(); it != sv->lru.end() && sv->table_bytes + bytes > sv->table_cap;) {
        TableEntry* e = it->get();
        if (e->in_use == 0 && e->ready) {
            cudaFreeAsync(e->base, st);
            sv->table_bytes -= e->bytes;
            sv->used -= e->bytes;
            sv->tables.erase(e->key);
            it = sv->lru.erase(it);
        } else {
            ++it;
        }
    }
    return sv->table_bytes + bytes <= sv->table_cap;
}

// Attach cached tables to the requests of a batch (server lock held).
static void attach_tables(Server* sv, Slot* sl) {
    for (auto& r : sl->reqs) {
        const std::string key = table_key(r->tool, r->proc);
        auto it = sv->tables.find(key);
        if (it != sv->tables.end()) {
            TableEntry* e = it->second.get();
            if (e->ready) {
                r->table = it->second;
                ++e->in_use;
                e->last_use = ++sv->tick;
                sv->lru.remove(it->second);
                sv->lru.push_back(it->second);
                ++sv->info.table_hits;
            } else {
                ++sv->info.table_misses;  // being built by a batch in flight: this one plans its own
            }
            continue;
        }
        ++sv->info.table_misses;
        const size_t bytes = align256(surface_table_bytes(r->tool, r->proc));
        if (!table_make_room(sv, bytes, sl->stream)) continue;
        if (sv->used + bytes > sv->budget) continue;
        char* base = nullptr;
        if (cudaMallocAsync((void**)&base, bytes, sl->stream) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        auto e = std::make_shared<TableEntry>();
        e->key = key;
        e->base = base;
        e->bytes = bytes;
        e->in_use = 1;
        e->last_use = ++sv->tick;
        sv->tables[key] = e;
        sv->lru.push_back(e);
        sv->table_bytes += bytes;
        sv->used += bytes;
        if (sv->used > sv->used_peak) sv->used_peak = sv->used;
        r->table = e;
        r->builds_table = true;
    }
}

// Launch one batch on a slot. Called without the server lock held.
static fsm_status launch_slot(Server* sv, Slot* sl) {
    const int n = (int)sl->reqs.size();
    std::vector<const fsm_tool_desc*> td(n);
    std::vector<const fsm_process_desc*> pd(n);
    std::vector<void*> hp(n);
    std::vector<TableRef> tr(n);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n; ++i) {
        Request* r = sl->reqs[i].get();
        td[i] = &r->tool;
        pd[i] = &r->proc;
        if (r->table) {
            tr[i].base = r->table->base;
            tr[i].ready = !r->builds_table;
        }
        int left = sv->fail_allocs.load();
        while (left > 0 && !sv->fail_allocs.compare_exchange_weak(left, left - 1)) {
        }
        if (left > 0) return fail(FSM_E_NOMEM, "device allocation failed (injected)");
        if ((e = cudaMallocAsync(&r->d_heights, r->map_bytes, sl->stream)) != cudaSuccess) {
            cudaGetLastError();
            r->d_heights = nullptr;
            return e == cudaErrorMemoryAllocation ? fail(FSM_E_NOMEM, "cudaMallocAsync (request heights)")
                                                  : cuda_fail(e, "cudaMallocAsync (request heights)");
        }
        hp[i] = r->d_heights;
    }
    if ((e = cudaEventRecord(sl->ev_start, sl->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    fsm_status rc = predict_batch_descs(sv->ctx, n, td.data(), pd.data(), hp.data(), sl->d_rough, nullptr,
                                        sl->stream, &sl->staging, tr.data());
    if (rc != FSM_OK) return rc;
    if ((e = cudaMemcpyAsync(sl->h_rough, sl->d_rough, sizeof(fsm_roughness_out) * n, cudaMemcpyDeviceToHost,
                             sl->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync (roughness)");
    if ((e = cudaEventRecord(sl->ev_end, sl->stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    sl->done.store(false);
    if ((e = cudaLaunchHostFunc(sl->stream, on_batch_done, sl)) != cudaSuccess)
        return cuda_fail(e, "cudaLaunchHostFunc");
    return FSM_OK;
}

// A request's cached tables are no longer needed by its launch (lock held).
// `built`: the launch completed, so tables it built are ready for others.
static void detach_table(Server* sv, Request* r, bool built, cudaStream_t st) {
    if (!r->table) return;
    TableEntry* e = r->table.get();
    --e->in_use;
    if (r->builds_table) {
        if (built) {
            e->ready = true;
        } else if (e->in_use == 0) {  // never built: drop it
            cudaFreeAsync(e->base, st);
            sv->table_bytes -= e->bytes;
            sv->used -= e->bytes;
            sv->tables.erase(e->key);
            sv->lru.remove(r->table);
        }
    }
    r->table.reset();
    r->builds_table = false;
}

static void log_batch(Server* sv, Slot* sl, int n) {
    fsm_batch_interval b{};
    b.slot = sl->index;
    b.n_requests = n;
    float t0 = 0.f, t1 = 0.f;
    if (cudaEventElapsedTime(&t0, sv->ev_origin, sl->ev_start) != cudaSuccess ||
        cudaEventElapsedTime(&t1, sv->ev_origin, sl->ev_end) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    b.t_start_ms = t0;
    b.t_end_ms = t1;
    if (sv->log.size() < kBatchLog) {
        sv->log.push_back(b);
    } else {
        sv->log[sv->log_next] = b;
    }
    sv->log_next = (sv->log_next + 1) % kBatchLog;
}

static void scheduler(Server* sv) {
    cudaSetDevice(sv->ctx->device);  // this thread's own device
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progressed = false;
        // reap finished batches
        for (auto& sp : sv->slots) {
            Slot* sl = sp.get();
            if (!sl->busy || !sl->done.load()) continue;
            const double td = sl->t_done.load();
            log_batch(sv, sl, (int)sl->reqs.size());
            ++sv->info.batches;
            for (size_t k = 0; k < sl->reqs.size(); ++k) {
                Request* r = sl->reqs[k].get();
                r->rough = sl->h_rough[k];
                r->t_done = td;
                detach_table(sv, r, true, sl->stream);
                sv->used -= r->extra_bytes;  // tables and scratch are gone; the map stays
                r->extra_bytes = 0;
                if (r->cancel) {  // cancelled while running: drop the map
                    r->status = FSM_E_CANCELLED;
                    cudaFreeAsync(r->d_heights, sl->stream);
                    r->d_heights = nullptr;
                    sv->used -= r->map_bytes;
                    ++sv->info.cancelled;
                } else {
                    r->status = FSM_OK;
                    ++sv->info.completed;
                }
            }
            sl->reqs.clear();
            sl->busy = false;
            progressed = true;
            sv->cv_done.notify_all();
        }
        // admit and launch on idle slots
        for (auto& sp : sv->slots) {
            Slot* sl = sp.get();
            if (sl->busy || sv->pending.empty()) continue;
            while (!sv->pending.empty() && (int)sl->reqs.size() < sv->max_batch) {
                auto& r = sv->pending.front();
                const size_t need = r->map_bytes + r->extra_bytes;
                if (sv->used + need > sv->budget) break;  // first in, first out
                sv->used += need;
                if (sv->used > sv->used_peak) sv->used_peak = sv->used;
                r->t_start = now_s();
                r->admitted = true;
                sl->reqs.push_back(r);
                sv->pending.pop_front();
            }
            if (sl->reqs.empty()) break;
            sl->busy = true;
            attach_tables(sv, sl);
            lk.unlock();
            fsm_status rc = launch_slot(sv, sl);
            lk.lock();
            if (rc != FSM_OK) {
                // nothing of this batch runs past its last successful enqueue;
                // wait for that before the memory goes back to the budget
                cudaStreamSynchronize(sl->stream);
                cudaGetLastError();
                for (auto& r : sl->reqs) {
                    r->status = r->cancel ? FSM_E_CANCELLED : rc;
                    r->t_done = now_s();
                    detach_table(sv, r.get(), false, sl->stream);
                    sv->used -= r->map_bytes + r->extra_bytes;
                    r->extra_bytes = 0;
                    if (r->d_heights) cudaFreeAsync(r->d_heights, sl->stream);
                    r->d_heights = nullptr;
                    ++(r->cancel ? sv->info.cancelled : sv->info.failed);
                }
                sl->reqs.clear();
                sl->busy = false;
                sv->cv_done.notify_all();
            }
            progressed = true;
        }
        if (!progressed) sv->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
    }
}

static void destroy_slots(Server* sv) {
    for (auto& s : sv->slots) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->ev_start) cudaEventDestroy(s->ev_start);
        if (s->ev_end) cudaEventDestroy(s->ev_end);
        s->staging.release();
        if (s->h_rough) cudaFreeHost(s->h_rough);
        if (s->d_rough) cudaFree(s->d_rough);
    }
    if (sv->ev_origin) cudaEventDestroy(sv->ev_origin);
}

}  // namespace fsm

using namespace fsm;

extern "C" {

fsm_status fsm_server_start(fsm_ctx* ctx, size_t budget_bytes, int32_t n_streams, int32_t max_batch) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    if (ctx->server) return fail(FSM_E_STATE, "a server is already running on this context");
    if (budget_bytes == 0 || n_streams < 1 || n_streams > 64 || max_batch < 1)
        return fail(FSM_E_INVALID, "budget > 0, 1 <= n_streams <= 64, max_batch >= 1");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    // keep freed stream-ordered memory cached in the pool for re-admission
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    Server* sv = new Server();
    sv->ctx = ctx;
    sv->budget = budget_bytes;
    sv->max_batch = max_batch;
    // planned tables may take up to 1/16 of the budget (at most 1 GiB)
    sv->table_cap = std::min(budget_bytes / 16, (size_t)1 << 30);
    for (int i = 0; i < n_streams; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->server = sv;
        sl->index = i;
        Slot* raw = sl.get();
        sv->slots.push_back(std::move(sl));
        if ((e = cudaStreamCreateWithFlags(&raw->stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&raw->ev_start)) != cudaSuccess ||
            (e = cudaEventCreate(&raw->ev_end)) != cudaSuccess ||
            (e = cudaMallocHost((void**)&raw->h_rough, sizeof(fsm_roughness_out) * max_batch)) != cudaSuccess ||
            (e = cudaMalloc((void**)&raw->d_rough, sizeof(fsm_roughness_out) * max_batch)) != cudaSuccess) {
            destroy_slots(sv);
            delete sv;
            return cuda_fail(e, "server slot setup");
        }
    }
    // device time origin of the batch log
    if ((e = cudaEventCreate(&sv->ev_origin)) != cudaSuccess ||
        (e = cudaEventRecord(sv->ev_origin, sv->slots[0]->stream)) != cudaSuccess ||
        (e = cudaEventSynchronize(sv->ev_origin)) != cudaSuccess) {
        destroy_slots(sv);
        delete sv;
        return cuda_fail(e, "server event setup");
    }
    sv->thr = std::thread(scheduler, sv);
    ctx->server = sv;
    return FSM_OK;
}

fsm_status fsm_server_stop(fsm_ctx* ctx) {
    if (!ctx || !ctx->server) return fail(FSM_E_STATE, "no server running");
    Server* sv = ctx->server;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_sched.notify_all();
    sv->thr.join();
    DeviceGuard dev_guard(ctx->device);
    for (auto& s : sv->slots) cudaStreamSynchronize(s->stream);
    cudaStream_t st0 = sv->slots[0]->stream;
    for (auto& kv : sv->all)
        if (kv.second->d_heights) cudaFreeAsync(kv.second->d_heights, st0);
    for (auto& e : sv->lru) cudaFreeAsync(e->base, st0);
    destroy_slots(sv);
    delete sv;
    ctx->server = nullptr;
    return FSM_OK;
}

fsm_status fsm_submit(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc, uint64_t* ticket) {
    if (!ctx || !tool || !proc || !ticket) return fail(FSM_E_INVALID, "NULL argument");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    auto r = std::make_shared<Request>();
    r->tool = tool->d;
    r->proc = proc->d;
    r->map_bytes = (size_t)proc->d.nx * (size_t)proc->d.ny * (proc->d.precision == FSM_FP64 ? 8 : 4);
    r->extra_bytes = surface_overhead_bytes(tool->d, proc->d);
    if (r->map_bytes + r->extra_bytes > sv->budget) return fail(FSM_E_NOMEM, "request larger than the budget");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        r->t_submit = now_s();
        sv->all[r->id] = r;
        sv->pending.push_back(r);
        *ticket = r->id;
        ++sv->info.submitted;
        const int depth = (int)sv->pending.size();
        if (depth > sv->info.queue_peak) sv->info.queue_peak = depth;
    }
    sv->cv_sched.notify_all();
    return FSM_OK;
}

fsm_status fsm_cancel(fsm_ctx* ctx, uint64_t ticket) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) return fail(FSM_E_STATE, "unknown ticket");
        Request* r = it->second.get();
        if (r->status != FSM_PENDING) return fail(FSM_E_STATE, "request already finished");
        if (r->cancel) return FSM_OK;
        r->cancel = true;
        if (!r->admitted) {  // still queued: it never reaches the device
            for (auto q = sv->pending.begin(); q != sv->pending.end(); ++q)
                if (q->get() == r) {
                    sv->pending.erase(q);
                    break;
                }
            r->status = FSM_E_CANCELLED;
            r->t_done = now_s();
            ++sv->info.cancelled;
        }
        // a running request finishes its batch; its map is dropped at completion
    }
    sv->cv_done.notify_all();
    sv->cv_sched.notify_all();
    return FSM_OK;
}

fsm_status fsm_poll(fsm_ctx* ctx, uint64_t ticket, int32_t timeout_ms, fsm_result* out) {
    if (!ctx || !out) return fail(FSM_E_INVALID, "NULL argument");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(FSM_E_STATE, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->status != FSM_PENDING; };
    if (!ready()) {
        if (timeout_ms == 0) return FSM_PENDING;
        if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
        else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return fail(FSM_E_TIMEOUT, "request not finished within timeout");
    }
    memset(out, 0, sizeof *out);
    out->d_heights = r->d_heights;
    out->precision = r->proc.precision;
    out->nx = r->proc.nx;
    out->ny = r->proc.ny;
    out->status = r->status;
    out->rough = r->rough;
    out->queue_s = r->admitted ? r->t_start - r->t_submit : r->t_done - r->t_submit;
    out->latency_s = r->t_done - r->t_submit;
    if (r->status == FSM_E_CANCELLED) return fail(FSM_E_CANCELLED, "request cancelled");
    if (r->status != FSM_OK) return fail((fsm_status)r->status, "request failed");
    return FSM_OK;
}

fsm_status fsm_release_result(fsm_ctx* ctx, uint64_t ticket) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->all.find(ticket);
        if (it == sv->all.end()) return fail(FSM_E_STATE, "unknown ticket");
        Request* r = it->second.get();
        if (r->status == FSM_PENDING) return fail(FSM_E_STATE, "request still running");
        if (r->d_heights) {
            DeviceGuard dev_guard(ctx->device);
            cudaFreeAsync(r->d_heights, sv->slots[0]->stream);
            sv->used -= r->map_bytes;
        }
        sv->all.erase(it);
    }
    sv->cv_sched.notify_all();
    return FSM_OK;
}

fsm_status fsm_server_stats(fsm_ctx* ctx, fsm_server_info* out) {
    if (!ctx || !out) return fail(FSM_E_INVALID, "NULL argument");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->info;
    out->queue_depth = (int32_t)sv->pending.size();
    out->bytes_in_use = sv->used;
    out->bytes_peak = sv->used_peak;
    out->table_bytes = sv->table_bytes;
    out->tables_cached = (int32_t)sv->tables.size();
    return FSM_OK;
}

fsm_status fsm_server_batches(fsm_ctx* ctx, fsm_batch_interval* out, int32_t capacity, int32_t* n) {
    if (!ctx || !n || (capacity > 0 && !out)) return fail(FSM_E_INVALID, "NULL argument");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    std::lock_guard<std::mutex> lk(sv->mu);
    const size_t have = sv->log.size();
    const size_t first = have < kBatchLog ? 0 : sv->log_next;  // oldest kept entry
    const size_t take = std::min(have, (size_t)std::max(capacity, 0));
    for (size_t i = 0; i < take; ++i) out[i] = sv->log[(first + have - take + i) % have];
    *n = (int32_t)take;
    return FSM_OK;
}

fsm_status fsm_server_inject_alloc_failures(fsm_ctx* ctx, int32_t count) {
    if (!ctx || count < 0) return fail(FSM_E_INVALID, "ctx is NULL or count < 0");
    Server* sv = ctx->server;
    if (!sv) return fail(FSM_E_STATE, "no server running");
    sv->fail_allocs.store(count);
    return FSM_OK;
}

}  // extern "C"
