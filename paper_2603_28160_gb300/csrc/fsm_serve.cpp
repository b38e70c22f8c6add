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
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fsm.h"
#include "fsm_host.h"

namespace fsm {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t id = 0;
    fsm_tool_desc tool{};
    fsm_process_desc proc{};
    size_t map_bytes = 0, extra_bytes = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    void* d_heights = nullptr;
    int status = FSM_PENDING;
    fsm_roughness_out rough{};
};

struct Slot {
    cudaStream_t stream = nullptr;
    PinnedSlot staging;
    fsm_roughness_out* h_rough = nullptr;  // pinned, max_batch entries
    fsm_roughness_out* d_rough = nullptr;  // device, max_batch entries
    std::vector<std::shared_ptr<Request>> reqs;
    bool busy = false;
    std::atomic<bool> done{false};
    std::atomic<double> t_done{0.0};
    struct Server* server = nullptr;
};

struct Server {
    fsm_ctx* ctx = nullptr;
    size_t budget = 0, used = 0;
    int max_batch = 1;
    std::vector<std::unique_ptr<Slot>> slots;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::thread thr;
    bool stop = false;
    uint64_t next_id = 1;
};

static void CUDART_CB on_batch_done(void* arg) {
    Slot* s = (Slot*)arg;
    s->t_done.store(now_s());
    s->done.store(true);
    s->server->cv_sched.notify_all();
}

// Launch one batch on a slot. Called without the server lock held.
static fsm_status launch_slot(Server* sv, Slot* sl) {
    const int n = (int)sl->reqs.size();
    std::vector<const fsm_tool_desc*> td(n);
    std::vector<const fsm_process_desc*> pd(n);
    std::vector<void*> hp(n);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n; ++i) {
        Request* r = sl->reqs[i].get();
        td[i] = &r->tool;
        pd[i] = &r->proc;
        if ((e = cudaMallocAsync(&r->d_heights, r->map_bytes, sl->stream)) != cudaSuccess)
            return cuda_fail(e, "cudaMallocAsync (request heights)");
        hp[i] = r->d_heights;
    }
    fsm_status rc = predict_batch_descs(sv->ctx, n, td.data(), pd.data(), hp.data(), sl->d_rough, nullptr,
                                        sl->stream, &sl->staging);
    if (rc != FSM_OK) return rc;
    if ((e = cudaMemcpyAsync(sl->h_rough, sl->d_rough, sizeof(fsm_roughness_out) * n, cudaMemcpyDeviceToHost,
                             sl->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync (roughness)");
    sl->done.store(false);
    if ((e = cudaLaunchHostFunc(sl->stream, on_batch_done, sl)) != cudaSuccess)
        return cuda_fail(e, "cudaLaunchHostFunc");
    return FSM_OK;
}

static void scheduler(Server* sv) {
    cudaSetDevice(sv->ctx->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progressed = false;
        // reap finished batches
        for (auto& sp : sv->slots) {
            Slot* sl = sp.get();
            if (!sl->busy || !sl->done.load()) continue;
            const double td = sl->t_done.load();
            for (size_t k = 0; k < sl->reqs.size(); ++k) {
                Request* r = sl->reqs[k].get();
                r->rough = sl->h_rough[k];
                r->t_done = td;
                r->status = FSM_OK;
                sv->used -= r->extra_bytes;  // tables and scratch are gone; the map stays
                r->extra_bytes = 0;
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
                r->t_start = now_s();
                sl->reqs.push_back(r);
                sv->pending.pop_front();
            }
            if (sl->reqs.empty()) break;
            sl->busy = true;
            lk.unlock();
            fsm_status rc = launch_slot(sv, sl);
            lk.lock();
            if (rc != FSM_OK) {
                for (auto& r : sl->reqs) {
                    r->status = rc;
                    sv->used -= r->map_bytes + r->extra_bytes;
                    r->extra_bytes = 0;
                    if (r->d_heights) cudaFreeAsync(r->d_heights, sl->stream);
                    r->d_heights = nullptr;
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

}  // namespace fsm

using namespace fsm;

extern "C" {

fsm_status fsm_server_start(fsm_ctx* ctx, size_t budget_bytes, int32_t n_streams, int32_t max_batch) {
    if (!ctx) return fail(FSM_E_INVALID, "ctx is NULL");
    if (ctx->server) return fail(FSM_E_STATE, "a server is already running on this context");
    if (budget_bytes == 0 || n_streams < 1 || n_streams > 64 || max_batch < 1)
        return fail(FSM_E_INVALID, "budget > 0, 1 <= n_streams <= 64, max_batch >= 1");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
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
    for (int i = 0; i < n_streams; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->server = sv;
        if ((e = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaMallocHost((void**)&sl->h_rough, sizeof(fsm_roughness_out) * max_batch)) != cudaSuccess ||
            (e = cudaMalloc((void**)&sl->d_rough, sizeof(fsm_roughness_out) * max_batch)) != cudaSuccess) {
            for (auto& s : sv->slots) {
                cudaStreamDestroy(s->stream);
                cudaFreeHost(s->h_rough);
                cudaFree(s->d_rough);
            }
            delete sv;
            return cuda_fail(e, "server slot setup");
        }
        sv->slots.push_back(std::move(sl));
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
    cudaSetDevice(ctx->device);
    for (auto& s : sv->slots) cudaStreamSynchronize(s->stream);
    for (auto& kv : sv->all)
        if (kv.second->d_heights) cudaFreeAsync(kv.second->d_heights, sv->slots[0]->stream);
    for (auto& s : sv->slots) {
        cudaStreamSynchronize(s->stream);
        cudaStreamDestroy(s->stream);
        s->staging.release();
        cudaFreeHost(s->h_rough);
        cudaFree(s->d_rough);
    }
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
    }
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
    out->queue_s = r->t_start - r->t_submit;
    out->latency_s = r->t_done - r->t_submit;
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
            cudaSetDevice(ctx->device);
            cudaFreeAsync(r->d_heights, sv->slots[0]->stream);
            sv->used -= r->map_bytes;
        }
        sv->all.erase(it);
    }
    sv->cv_sched.notify_all();
    return FSM_OK;
}

}  // extern "C"
