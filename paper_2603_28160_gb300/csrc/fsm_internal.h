// fsm_internal.h -- launchers shared by the C ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>

#include "../../include/fsm.h"
#include "fsm_device.cuh"

namespace fsm {

// Build tables and derived values of n surfaces (one block each). If `one`
// is not NULL it is copied into d_surfs[0] first (n must be 1).
// Planning of n surfaces (one: a single surface passed by value). Each
// surface gets up to kPlanParts blocks, as many as its largest
// (edge points + phases) work calls for while n x blocks stays within a few
// waves of the GPU's sm_count SMs; max_work is taken from `one` when given.
cudaError_t launch_plan(Surface* d_surfs, int n, const Surface* one, int max_work, int sm_count, cudaStream_t st);

size_t sweep_smem_bytes(int precision, int tile_x, int tile_y, int threads);
size_t sweep_static_bytes();  // static shared memory of the sweep kernels
int sweep_blocks_per_sm(int precision, int threads, size_t smem);
cudaError_t sweep_allow_smem(size_t max_bytes);
// phase_form: surfaces whose runs come back for many revolutions share
// per-phase work (see phase_form_pays); tilt: some surface is fed off the X
// axis (the launch then takes the phase-capable tilted instantiation).
cudaError_t launch_sweep_shaped(int precision, const Surface* d_surfs, int n_surf,
                                const int* d_tile_base, int total_tiles, int* d_queue,
                                long long* d_counters, int grid, int threads, size_t smem,
                                cudaStream_t st, bool phase_form, bool tilt);

// A feed direction off the X axis (not a multiple of 360 degrees).
inline bool feed_tilted(const fsm_process_desc& p) { return fmod(p.feed_dir_deg, 360.0) != 0.0; }

// Whether the sweep is launched in the instantiation that chooses between
// the item and the phase form per task (otherwise every task takes the item
// form). FP32 maps: when a tile is at least one and a half feeds per
// revolution wide, so that the runs of one tile come back for more than one
// revolution (measured on GB300 with 16 warps on 152 KB tiles: the ball
// raster at two feeds per tile 0.967 ms against 0.983 ms item by item; the
// side wall and the flat-end floor, at two to four, are faster by phase).
// FP64 maps always: their FP64 height is computed once per phase in the
// phase form, and the per-task choice keeps runs of few revolutions item by
// item (ball raster FP64 4.55 -> 3.57 ms with 512x32 tiles, 8 mm floor
// 79.6 -> 55.0 ms).
inline bool phase_form_pays(const fsm_tool_desc& t, const fsm_process_desc& p, int tile_x, int form = 0) {
    if (feed_tilted(p)) return false;
    if (form == FSM_FORM_PHASE) return true;
    if (form == FSM_FORM_ITEM) return false;
    if (p.precision == FSM_FP64) return true;
    const double feeds = (double)tile_x * p.pitch / ((double)t.n_teeth * p.fz);
    return feeds >= 1.5;
}

// Trajectory map of one planned surface: argmin table d_jmin (S * n_teeth
// int32 of scratch), then n_records = total steps * n_teeth records.
cudaError_t launch_trajectory(const Surface* d_surf, int S, int n_teeth, long long n_records, int32_t* d_jmin,
                              fsm_traj_point* d_out, cudaStream_t st);

// Roughness of a set of maps of one precision. Map j is cut into
// ceil(n/kChunk) chunks; d_chunk_base[j] is its first chunk (n_jobs+1
// entries). d_part: rough_part_doubles(total_chunks, n_jobs, max_profiles)
// doubles of scratch; d_sync:
// rough_sync_bytes(n_jobs) of scratch (8-byte aligned; cleared by the call).
// max_profiles = the largest n_rows + n_cols of any job. One memset and two
// launches.
constexpr size_t kChunk = 32768;
struct RoughJob {
    const void* h;
    size_t n;
    int nx, ny, n_rows, n_cols;
    fsm_roughness_out* out;
};
size_t rough_sync_bytes(int n_jobs);
// Doubles of roughness partials: 7 per chunk, then 4 per profile segment
// (5 segments of max_profiles profiles per job).
size_t rough_part_doubles(int total_chunks, int n_jobs, int max_profiles);
cudaError_t launch_roughness_jobs(int precision, const RoughJob* d_jobs, int n_jobs, const int* d_chunk_base,
                                  int total_chunks, int max_profiles, double* d_part, void* d_sync,
                                  cudaStream_t st);
// Moment partials of n cells about `about` (see fsm_moment_partials):
// d_ws of moment_ws_bytes(n) bytes, 8 doubles to d_out; two launches.
size_t moment_ws_bytes(size_t n);
cudaError_t launch_moments(int precision, const void* d_h, size_t n, double about, double* d_ws, double* d_out,
                           cudaStream_t st);
// One map; d_ws of roughness_one_ws_bytes(n) bytes (256-aligned).
size_t roughness_one_ws_bytes(size_t n);
cudaError_t launch_roughness_one(int precision, const RoughJob& jb, char* d_ws, cudaStream_t st);

}  // namespace fsm
