// fsm_host.h -- host-side handles and helpers shared by the C ABI files.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <map>
#include <mutex>
#include <string>

#include "../../include/fsm.h"
#include "fsm_device.cuh"

struct fsm_tool {
    fsm_tool_desc d;
};
struct fsm_process {
    fsm_process_desc d;
};

namespace fsm {
struct Server;
}

struct fsm_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::mutex mu;
    fsm::Server* server = nullptr;
    // autotuned sweep shapes: workload signature -> (tile_x, tile_y, ctas_per_sm, threads)
    std::map<std::string, std::array<int, 4>> tuned;
    // resident sweep CTAs per SM: (precision, threads, shared bytes) -> count
    std::map<std::array<long long, 3>, int> occupancy;
    // device address of the allocation-free roughness scratch (first use)
    char* noalloc_scratch = nullptr;
};

namespace fsm {

// A pinned host staging buffer whose reuse waits for its last copy.
struct PinnedSlot {
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    cudaError_t ensure(size_t bytes) {
        cudaError_t e = cudaSuccess;
        if (!done) {
            if ((e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess) return e;
        } else if ((e = cudaEventSynchronize(done)) != cudaSuccess) {
            return e;
        }
        if (cap < bytes) {
            if (host) cudaFreeHost(host);
            host = nullptr;
            cap = 0;
            if ((e = cudaMallocHost(&host, bytes + bytes / 2)) != cudaSuccess) return e;
            cap = bytes + bytes / 2;
        }
        return e;
    }
    void release() {
        if (done) cudaEventSynchronize(done);
        if (host) cudaFreeHost(host);
        if (done) cudaEventDestroy(done);
        host = nullptr;
        done = nullptr;
        cap = 0;
    }
};

// Makes ctx's device current for the duration of an entry point and gives
// the calling thread its previous current device back on every return, so a
// host thread that drives several GPUs keeps its own choice of device.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != device) {
            err = cudaSetDevice(device);
            changed = err == cudaSuccess && prev >= 0;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

fsm_status fail(fsm_status st, const std::string& msg);
fsm_status cuda_fail(cudaError_t e, const char* what);

struct Shape {
    int tile_x, tile_y, threads;
};

size_t align256(size_t v);
// Key of the autotuner's table for a tool/process pair.
std::string tune_key(const fsm_tool_desc& t, const fsm_process_desc& p);
// Sweep shape: the caller's override, else the default ladder step for this
// precision given the tiles of the surfaces in `group` (may be NULL); with
// `tools` (one per group entry), a lone surface of this precision gets a
// tile width aligned to its feed per revolution.
Shape pick_shape(const fsm_process_desc& p, const fsm_predict_opts* o, const fsm_process_desc* const* group = nullptr,
                 int n_group = 0, int sm_count = 0, const fsm_tool_desc* const* tools = nullptr);
// Fill a device plan from the descriptors. Table pointers are laid out from
// `base`; returns the table bytes (call with base = NULL to size).
size_t fill_surface(const fsm_tool_desc& t, const fsm_process_desc& p, const Shape& sh, Surface* s,
                    char* base);
fsm_status sweep_config(fsm_ctx* ctx, int precision, const Shape& sh, size_t* smem, int* blocks_per_sm);
// Validate the caller's prediction overrides (NULL = defaults).
// Options valid (the surfaces of the call, for checks that need them).
fsm_status check_opts(const fsm_predict_opts* o, const fsm_process_desc* const* procs, int n);
fsm_status predict_one(fsm_ctx* ctx, const fsm_tool_desc& t, const fsm_process_desc& p, void* d_heights,
                       const fsm_predict_opts* opts, cudaStream_t st);
fsm_status check_fp32_band(const fsm_tool_desc& t, const fsm_process_desc& p, const Shape& sh);
fsm_status trajectory_one(fsm_ctx* ctx, const fsm_tool_desc& t, const fsm_process_desc& p, fsm_traj_point* d_out,
                          int64_t capacity, cudaStream_t st);
fsm_status roughness_one(fsm_ctx* ctx, const void* d_h, int precision, int nx, int ny, int n_rows, int n_cols,
                         fsm_roughness_out* d_out, cudaStream_t st);

// Device bytes one surface needs beyond its height map (tables + scratch).
size_t surface_overhead_bytes(const fsm_tool_desc& t, const fsm_process_desc& p);

// Device tables of one surface held outside a batch (a server's table
// cache): `base` is laid out as fill_surface lays out a surface's tables;
// `ready` says they were built by an earlier, completed launch (the planning
// kernels then skip them), else this launch builds them there.
struct TableRef {
    char* base = nullptr;
    bool ready = false;
};

// One-shot batch on stream-ordered scratch; `slot` (optional) stages the
// upload in pinned memory; `trefs` (optional, one per surface) places
// surfaces' tables outside the batch's scratch.
fsm_status predict_batch_descs(fsm_ctx* ctx, int n, const fsm_tool_desc* const* td,
                               const fsm_process_desc* const* pd, void* const* d_heights,
                               fsm_roughness_out* d_rough, const fsm_predict_opts* opts, cudaStream_t st,
                               PinnedSlot* slot, const TableRef* trefs = nullptr);

// Bytes of a surface's device tables (the layout fill_surface gives).
size_t surface_table_bytes(const fsm_tool_desc& t, const fsm_process_desc& p);

}  // namespace fsm
