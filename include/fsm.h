/*
 * fsm.h -- C ABI of the GB300 forward-solution-method (FSM) surface generator.
 *
 * The library predicts the 3D topography left by a milling tool (Section 2 of
 * "An efficient open-source framework for high-fidelity 3D surface topography
 * and roughness prediction in milling", arXiv 2603.28160) and reduces it to
 * roughness indicators (Section 4.1.2). Every step of the computation runs in
 * CUDA kernels for sm_103a; the host only validates descriptors and launches.
 *
 * Conventions shared by all entry points
 *   - Lengths in mm, angles in degrees.
 *   - Height maps are row-major H[ny][nx]: row k is along +Y_W (step-over),
 *     column i along +X_W (feed). Cell (i,k) covers
 *     [x0 + i*pitch, x0 + (i+1)*pitch) x [y0 + k*pitch, y0 + (k+1)*pitch)
 *     (the sampling boundaries of Eq. eq_sampling_boundaries, read as
 *     half-open so that every point belongs to exactly one cell).
 *   - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *     data_ptr()); `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream). All enqueueing calls are asynchronous on that stream.
 *   - Every function returns an fsm_status; no C++ exception crosses the ABI.
 *     After an error, fsm_last_error(ctx) returns a message for the calling
 *     thread's most recent failure on that context.
 *   - Handles are opaque and owned by the library; descriptors are copied at
 *     creation, so the caller may free them afterwards.
 */
#ifndef FSM_H
#define FSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FSM_MAX_TEETH 16
#define FSM_MAX_PROFILES 16

typedef enum {
    FSM_OK = 0,
    FSM_PENDING = 1,          /* fsm_poll: the request has not finished */
    FSM_E_INVALID = -1,       /* a descriptor or argument failed validation */
    FSM_E_NOMEM = -2,         /* device memory or the admission budget ran out */
    FSM_E_CUDA = -3,          /* a CUDA runtime call failed */
    FSM_E_TIMEOUT = -4,       /* fsm_poll waited timeout_ms without completion */
    FSM_E_CANCELLED = -5,     /* the request was cancelled */
    FSM_E_STATE = -6          /* wrong call order (e.g. unknown ticket) */
} fsm_status;

enum { FSM_TOOL_FLAT = 0, FSM_TOOL_BALL = 1, FSM_TOOL_INSERT = 2, FSM_TOOL_TORUS = 3 };
enum { FSM_SURFACE_FLOOR = 0, FSM_SURFACE_WALL = 1 };
enum { FSM_PASS_ONE_WAY = 0, FSM_PASS_ZIGZAG = 1 };
enum { FSM_FP64 = 0, FSM_FP32 = 1 };

typedef struct fsm_ctx fsm_ctx;
typedef struct fsm_tool fsm_tool;
typedef struct fsm_process fsm_process;

/* Cutting tool (Section 2.1, Eq. eq_point_p_equation and
 * eq_cutting_edge_to_tool, generalised from round inserts to end mills).
 *   kind      FSM_TOOL_FLAT: bottom edge (h = 0, r in [0, D/2], n_end points)
 *             plus flank (r = D/2, h in [0, ap], n_edge points).
 *             FSM_TOOL_BALL: n_edge points uniform in polar angle on the
 *             sphere of radius D/2, over the cap that can reach the depth of
 *             cut for the process's lead/tilt.
 *   helix_deg per tooth; the edge at height h lags the tooth position by
 *             h tan(helix) / (D/2) radians against the rotation.
 *   tooth_deg angular position of each tooth (tooth K sits -tooth_deg[K]
 *             from the spindle reference, the sign of Eq. eq_tool_to_spindle).
 *             FSM_TOOL_INSERT: the paper's face mill with round indexable
 *             inserts of radius insert_radius (Eq. eq_point_p_equation):
 *             n_edge points on the insert's lower semicircle with
 *             l uniform in [-dL, dL], dL = max(sqrt(R^2 - (R-ap)^2),
 *             fz / (2 cos rake_f)) capped at R (Eq. eq_tool_point_p_equation);
 *             placed by Eq. eq_cutting_edge_to_tool: radial/axial rake
 *             rotation, lowest point at radius D/2 + K eps_r and height
 *             K eps_a for insert K = 0..n_teeth-1 (the paper's K-1).
 *             FSM_TOOL_TORUS (an extension): bull-nose end mill with corner
 *             radius corner_radius = rc: n_end bottom points at h = 0, r
 *             uniform in [0, D/2 - rc], then n_edge points uniform in arc
 *             length along the corner arc (centre (D/2 - rc, rc)) and the
 *             flank, from the bottom up to height ap.
 *   runout    spindle-axis offset of radius runout_mm at runout_phase_deg in
 *             the rotating frame.
 * Validation: 1 <= n_teeth <= 16, n_edge >= 2, n_end == 0 or >= 2 (flat,
 * torus), n_end == 0 (ball, insert), D > 0, runout >= 0, insert_radius > 0
 * (insert), 0 < corner_radius <= D/2 (torus), all values finite. helix_deg
 * is ignored for inserts. */
typedef struct {
    int32_t kind;
    int32_t n_teeth;
    int32_t n_edge;
    int32_t n_end;
    double diameter;
    double helix_deg[FSM_MAX_TEETH];
    double tooth_deg[FSM_MAX_TEETH];
    double runout_mm;
    double runout_phase_deg;
    double insert_radius;
    double rake_f_deg;
    double rake_p_deg;
    double eps_r_mm;
    double eps_a_mm;
    double corner_radius;
} fsm_tool_desc;

/* Cutting conditions, tool path and sampling grid (Sections 2.1-2.2).
 *   Time is discretised by the spindle angle: step s has phase index
 *   m = s mod S (S = 360/rot_step_deg, an integer) and spindle angle
 *   phase0_deg + rot_sense * m * rot_step_deg. The feed per step is
 *   n_teeth * fz / S along +X_W (Eq. eq_spindle_to_workpiece).
 *   Pass p (0 <= p < n_passes) covers global steps
 *   [p*steps_per_pass, (p+1)*steps_per_pass); its tool reference point starts
 *   at (pass_x0, pass_y0 + p*ae) and the spindle keeps turning between
 *   passes. The tool reference height is chosen so the lowest position any
 *   edge point reaches in a revolution is stock_z - ap.
 *   lead_deg leans the tool axis toward +X_W, tilt_deg toward +Y_W.
 *   precision FSM_FP64 (double heights: the FP64 height of every point and
 *   the cell its FP64 pose falls in, i.e. the map of an all-FP64 sweep; the
 *   cell is decided from FP32 tile-local coordinates where an error bound
 *   proves it, else from the FP64 pose) or FSM_FP32 (float heights: the
 *   FP32 height of every point in the cell its FP64 pose falls in, decided
 *   the same way; FP64 for the spindle phase, the path position and
 *   near-boundary re-binning). Neither map depends on the launch shape.
 *   surface FSM_SURFACE_FLOOR: the map covers x (columns) and y (rows) from
 *   (x0, y0), height z, un-machined at stock_z. FSM_SURFACE_WALL (an
 *   extension; the paper maps floors only): the side wall the flank leaves
 *   on the +Y side of a single pass, sampled over x (columns) and z (rows)
 *   from (x0, y0 = lowest z), height -y (the wall's outward normal is -Y),
 *   un-machined at y = wall_y, so cells keep -wall_y until cut. The tool
 *   reference height is the same as for the floor (stock_z - ap lowest).
 *   pass_mode FSM_PASS_ONE_WAY: every pass runs along +X from pass_x0;
 *   FSM_PASS_ZIGZAG: odd passes run back along -X over the same stretch
 *   (their step n is where step steps_per_pass-1-n of an even pass is).
 *   feed_dir_deg (an extension; the paper feeds along one axis): the feed
 *   direction in the XY plane, degrees counter-clockwise from +X. The tool
 *   path and the tool of the feed_dir_deg = 0 process (lead, tilt and
 *   spindle phase included) are turned by this angle about the vertical
 *   through (pass_x0, pass_y0): passes run along (cos, sin) and step over
 *   along (-sin, cos); the grid stays axis-aligned. A multiple of 360 is the
 *   +X feed itself. Floors only.
 * Validation: fz, ap, pitch > 0; 360/rot_step_deg integral; rot_sense = +-1;
 * n_passes >= 1 (== 1 for a wall); steps_per_pass >= 1;
 * n_passes*steps_per_pass < 2^31; 1 <= nx, ny <= 65535*256; finite values;
 * feed_dir_deg a multiple of 360 for a wall. rpm only labels time.
 * feed_dir_deg was added after `reserved`; zero it for the +X feed. */
typedef struct {
    double fz;
    double rpm;
    double rot_step_deg;
    double phase0_deg;
    int32_t rot_sense;
    int32_t n_passes;
    double ap;
    double lead_deg;
    double tilt_deg;
    double ae;
    double pass_x0;
    double pass_y0;
    int64_t steps_per_pass;
    double stock_z;
    double x0;
    double y0;
    double pitch;
    int32_t nx;
    int32_t ny;
    int32_t precision;
    int32_t surface;
    double wall_y;
    int32_t pass_mode;
    int32_t reserved;
    double feed_dir_deg;
} fsm_process_desc;

/* Optional launch overrides, counters and timing for the prediction calls.
 *   tile_x, tile_y    shared-memory tile in cells (0 = library default;
 *                     tile_x a multiple of 4)
 *   block_threads     threads per CTA, a multiple of 32 in 64..512 (0 = default)
 *   ctas_per_sm       cap on resident CTAs per SM (0 = as many as fit)
 *   d_counters        NULL, or device int64_t[4] the sweep ADDS to:
 *                     [0] edge-point poses evaluated (the FP32 sweep's
 *                         phase form skips revolutions that cannot reach a
 *                         tile, so this count depends on the form used),
 *                     [1] cutting evaluations: inside the patch and below the
 *                         stock surface (the points the per-cell minimum runs
 *                         over); exact in FP64, within ~1e-5 relative in FP32
 *                         (a point within FP32 error of a tile edge is counted
 *                         by its FP32 cell),
 *                     [2] cutting points re-binned in FP64 (FP32 path),
 *                     [3] shared-memory atomic updates issued.
 *   sweep_events      NULL or two cudaEvent_t (as void*) recorded on the
 *                     stream just before and just after the sweep launch(es),
 *                     to time the sweep kernel alone.
 *   sweep_form        how each (pass, tooth, 32-point group) task of the
 *                     sweep walks the steps of its time window (both forms
 *                     evaluate exactly the same points with the same
 *                     arithmetic, so the map does not depend on the choice):
 *                     FSM_FORM_AUTO (0): chosen per task by the library;
 *                     FSM_FORM_ITEM (1): step by step;
 *                     FSM_FORM_PHASE (2): spindle phase by phase, visiting
 *                     only the revolutions of each phase that can reach the
 *                     tile.
 *   d_form_tasks      NULL or device int64_t[2] the sweep ADDS to: tasks
 *                     walked in the item form [0] and in the phase form [1].
 * Fields after sweep_events were added later; zero them for the defaults. */
typedef struct {
    int32_t tile_x;
    int32_t tile_y;
    int32_t block_threads;
    int32_t ctas_per_sm;
    int64_t* d_counters;
    void* sweep_events[2];
    int32_t sweep_form;
    int32_t reserved;
    int64_t* d_form_tasks;
} fsm_predict_opts;

enum { FSM_FORM_AUTO = 0, FSM_FORM_ITEM = 1, FSM_FORM_PHASE = 2 };

/* Areal (ISO 25178-2) and line (ISO 4287) roughness of one height map,
 * Section 4.1.2. Mean plane = arithmetic mean; no form removal, no S/L
 * filter. Ssk = Sku = NaN when Sq == 0. Profiles: n_rows rows at
 * k_r = floor((2r+1) ny / (2 n_rows)) (along the feed) and n_cols columns at
 * i_c = floor((2c+1) nx / (2 n_cols)) (across the feed). Ra = mean |z - mean|
 * of the profile; Rz = mean over 5 consecutive segments
 * [floor(q L/5), floor((q+1) L/5)) of (max - min), NaN when L < 5. */
typedef struct {
    double n, mean, zmin, zmax;
    double Sa, Sq, Sp, Sv, Sz, Ssk, Sku;
    int32_t n_rows, n_cols;
    int32_t row_index[FSM_MAX_PROFILES], col_index[FSM_MAX_PROFILES];
    double Ra_row[FSM_MAX_PROFILES], Rz_row[FSM_MAX_PROFILES];
    double Ra_col[FSM_MAX_PROFILES], Rz_col[FSM_MAX_PROFILES];
} fsm_roughness_out;

/* ---------------------------------------------------------------------- */
/* Context and handles                                                     */
/* ---------------------------------------------------------------------- */

/* Create a context bound to CUDA device `device`. Fails with FSM_E_CUDA if
 * the device cannot be used (no GPU, or the library was not built for it).
 * Every entry point taking a context makes its device current for the call
 * and restores the calling thread's current device before returning. A
 * context belongs to the device's CUDA primary context as it was when the
 * context was created: after cudaDeviceReset, destroy and recreate it. */
fsm_status fsm_create_context(int device, fsm_ctx** out);
fsm_status fsm_destroy_context(fsm_ctx* ctx);

/* Message for the calling thread's last failure on ctx (never NULL; ctx may
 * be NULL for failures of fsm_create_context). Valid until the next call. */
const char* fsm_last_error(fsm_ctx* ctx);

/* Validate and copy a tool description (Section 3.2 "tool geometry module":
 * the geometry is fixed at construction). */
fsm_status fsm_create_tool(fsm_ctx* ctx, const fsm_tool_desc* desc, fsm_tool** out);
fsm_status fsm_destroy_tool(fsm_ctx* ctx, fsm_tool* tool);

/* Validate and copy cutting conditions, tool path and grid. */
fsm_status fsm_set_process(fsm_ctx* ctx, const fsm_process_desc* desc, fsm_process** out);
fsm_status fsm_destroy_process(fsm_ctx* ctx, fsm_process* proc);

/* ---------------------------------------------------------------------- */
/* Single surface                                                          */
/* ---------------------------------------------------------------------- */

/* Predict one height map: build the edge, phase and path tables on the
 * device (Section 2.2), sweep every edge point of every time step into a
 * shared-memory tile of the grid keeping the per-cell minimum height
 * (Section 2.3, Eq. eq_sampling_boundaries), and store the tiles.
 *   d_heights  caller-owned device buffer of ny*nx doubles (FSM_FP64) or
 *              floats (FSM_FP32), 16-byte aligned for vector stores (any
 *              alignment works, slower). Every cell is written; cells no edge
 *              point reaches keep stock_z.
 *   opts       NULL for defaults.
 * FSM_E_INVALID for an FP32 map whose pitch is too fine for FP32 tile-local
 * binning with this tool and pass (worst-case FP32 error bound of 0.45 cell
 * or more: about 20 nm and below for a 10 mm tool); FP64 maps have no such
 * limit. The same holds for every FP32 surface of a batch.
 * Scratch: stream-ordered device allocations (cudaMallocAsync) freed on the
 * same stream. Asynchronous; errors of the enqueue are returned, kernel
 * faults surface at the next synchronisation. */
fsm_status fsm_predict_surface(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc,
                               void* d_heights, const fsm_predict_opts* opts, void* stream);

/* One record of a trajectory map (32 bytes). */
typedef struct {
    double x, y, z;   /* workpiece coordinates of the lowest edge point (mm) */
    int32_t j;        /* its index along the edge (tool-description order) */
    int32_t tooth;    /* K, 0-based */
} fsm_traj_point;

/* Trajectory map (Section 3.1, trajectory computation module; the paper's
 * trajectory-map figures of Section 4.2): at every time step s of the tool
 * path (s = pass * steps_per_pass + local step) and for every tooth K, the
 * edge point of lowest workpiece z and its coordinates, computed in FP64 for
 * either process precision with the same pose arithmetic as the FP64 map.
 * Among points of equal z the first in edge order is reported.
 *   d_out      caller-owned device array of at least n_passes *
 *              steps_per_pass * n_teeth records, record s * n_teeth + K.
 *   capacity   records d_out can hold; fewer than needed -> FSM_E_INVALID.
 * Asynchronous on `stream`; stream-ordered scratch (tables and one int32 per
 * spindle phase and tooth). */
fsm_status fsm_predict_trajectory(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc,
                                  fsm_traj_point* d_out, int64_t capacity, void* stream);

/* Number of trajectory records of a tool/process pair (host only). */
fsm_status fsm_trajectory_records(const fsm_tool* tool, const fsm_process* proc, int64_t* n);

/* Autotuner (no counterpart in the paper, whose CPU loops have no launch
 * shape): times up to max_candidates (0 = all) sweep configurations -- tile
 * shape and resident CTAs per SM -- on this tool and process, writing into
 * d_heights, and returns the fastest in *best (d_counters and sweep_events
 * cleared) with its sweep time in *best_ms (host). The choice is recorded in
 * the context: later fsm_predict_surface calls with the same tool/process
 * shape (precision, tool kind, teeth, edge points, steps per revolution,
 * grid size and pitch) and no tile override use it. Synchronises the stream.
 * The map contents afterwards are those of the last candidate run (all
 * candidates compute the same map, bit for bit, in either precision). */
fsm_status fsm_autotune(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc, void* d_heights,
                        int32_t max_candidates, fsm_predict_opts* best, float* best_ms, void* stream);

/* Roughness of a device height map (FSM_FP64 doubles or FSM_FP32 floats),
 * computed on the device to FP64 accuracy (double-float sums on the FP32
 * pipes; each deviation of an FP64 map formed in FP64) with a fixed
 * reduction order (results do not depend on launch timing). Writes one fsm_roughness_out to DEVICE memory
 * d_out (caller-owned). 0 <= n_rows, n_cols <= 16. Asynchronous. */
fsm_status fsm_roughness(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx,
                         int32_t ny, int32_t n_rows, int32_t n_cols, fsm_roughness_out* d_out,
                         void* stream);

/* Roughness without any device allocation (the paper has no counterpart:
 * this exists for callers of the library that must not allocate device
 * memory once they are running -- a host that has already handed all device
 * memory to its own pool, a control loop with a fixed memory footprint, or
 * code that may not call cudaMalloc/cudaMallocAsync at all). Same result as
 * fsm_roughness, computed by the same kernels, but the per-chunk partial
 * sums live in a fixed array of about 0.9 MiB that the library reserves in
 * device memory on every GPU that loads it, until the process exits.
 *   Limit: nx * ny <= 536870912 (2^29) cells; larger maps fail with
 *          FSM_E_INVALID and a message saying so.
 *   The first call on a context looks the array's device address up on
 *   the context's device (with it made current) and keeps it in the
 *   context; make that first call before any stream capture. (After a
 *   cudaDeviceReset the address may change: recreate the context, as for
 *   every other entry point.)
 *   All calls on a device share the one array: calls whose kernels overlap on
 *   the GPU (e.g. on two streams) race and give wrong results; order them on
 *   one stream or synchronise between them. The array keeps the last call's
 *   contents; no part of it needs to start at zero (every word a call reads
 *   is written earlier in the same call).
 * Arguments as for fsm_roughness; no cudaMalloc, cudaFree or allocating
 * library call is made. */
fsm_status fsm_roughness_noalloc(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx,
                                 int32_t ny, int32_t n_rows, int32_t n_cols,
                                 fsm_roughness_out* d_out, void* stream);

/* Moment partials of a device height map, or of one row band of a map that
 * several devices computed band by band (each band is the map's rows
 * [k0, k1): the same process with y0 + k0 pitch and k1 - k0 rows). With
 * d = z - about, writes 8 doubles to DEVICE d_out: [0] cells, [1] sum d,
 * [2] min z, [3] max z, [4] sum |d|, [5] sum d^2, [6] sum d^3, [7] sum d^4,
 * each summed in a fixed order (FP64 maps in FP64; FP32 maps: d as an exact
 * float pair, terms summed in double-float). Combining bands: add [0], [1]
 * (about a common value) and take min/max of [2], [3] over the bands; the
 * map's mean is about + sum d / n; a second call per band with about = that
 * mean gives the bands' shares of the central sums of Section 4.1.2's Sa,
 * Sq, Ssk, Sku (added over the bands). Stream-ordered scratch of 64 bytes
 * per 32768 cells. Asynchronous on `stream`. (An extension: the paper's
 * method runs on one CPU.) */
fsm_status fsm_moment_partials(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx, int32_t ny,
                               double about, double* d_out, void* stream);

/* ISO 16610-61 areal Gaussian filtering of a device height map (an
 * extension for comparing predictions with measured surfaces: the paper's
 * profilometer applies an S-filter of 10 um and an L-filter of 0.8 mm,
 * Section 4.1.1).
 *   Weighting function s(x) = exp(-pi (x / (alpha lambda))^2) / (alpha
 *   lambda), alpha = sqrt(ln 2 / pi) (50 % transmission at lambda), sampled
 *   at the cells t * pitch for |t| <= floor(lambda / pitch), with the
 *   zero-order end correction: each output divides by the sum of the weights
 *   that fall inside the map. Applied along rows and columns (the areal
 *   function is separable).
 *   The S-filter gives the S-F surface S = s_{lambda_s} * H (S = H when
 *   lambda_s == 0); d_out = S - s_{lambda_c} * S, the SL-surface (d_out = S
 *   when lambda_c == 0).
 *   precision  FSM_FP64: doubles in and out, sums in double-float arithmetic
 *              (about 1e-14 relative); FSM_FP32: floats, FP32 sums.
 *   d_out      caller-owned device buffer of ny*nx values (row-major like
 *              d_heights), not d_heights itself.
 * Validation: nx, ny >= 1; pitch > 0; lambda_s, lambda_c >= 0; all finite;
 * lambda / pitch <= 4096. Scratch: three map-sized stream-ordered device
 * buffers. Asynchronous on `stream`. */
fsm_status fsm_filter(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx, int32_t ny,
                      double pitch, double lambda_s, double lambda_c, void* d_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched prediction                                                      */
/* ---------------------------------------------------------------------- */

/* Predict n surfaces of mixed tools, grids and precisions in one persistent
 * launch (plus one planning launch and, if d_rough != NULL, the roughness
 * launches). tools[i], procs[i] describe surface i; d_heights[i] is a HOST
 * array of n device pointers (each sized as in fsm_predict_surface);
 * d_rough NULL or a device array of n fsm_roughness_out (10 row and 10 column
 * profiles each). Work is distributed over (surface, tile) items by a device
 * queue. Asynchronous; stream-ordered scratch. */
fsm_status fsm_predict_batch(fsm_ctx* ctx, int32_t n, const fsm_tool* const* tools,
                             const fsm_process* const* procs, void* const* d_heights,
                             fsm_roughness_out* d_rough, const fsm_predict_opts* opts,
                             void* stream);

/* A prepared batch for repeated launches and CUDA-graph capture: the
 * descriptors, table space and scratch of n surfaces are laid out once in a
 * device buffer owned by the batch (synchronous upload at creation).
 * fsm_batch_run then enqueues only a memset and kernel launches (planning,
 * the persistent sweep per precision, roughness), so a stream capture of it
 * replays as a CUDA graph. Runs of one batch must not overlap in time (they
 * share its scratch). Arguments as for fsm_predict_batch. */
typedef struct fsm_batch fsm_batch;
fsm_status fsm_batch_create(fsm_ctx* ctx, int32_t n, const fsm_tool* const* tools,
                            const fsm_process* const* procs, void* const* d_heights,
                            fsm_roughness_out* d_rough, const fsm_predict_opts* opts,
                            fsm_batch** out);
fsm_status fsm_batch_run(fsm_ctx* ctx, fsm_batch* batch, void* stream);
fsm_status fsm_batch_destroy(fsm_ctx* ctx, fsm_batch* batch);

/* ---------------------------------------------------------------------- */
/* Served requests (continuous batching)                                   */
/* ---------------------------------------------------------------------- */

/* Start a request server on ctx. Requests are admitted while the device
 * memory they need (height map + tables + scratch) fits in budget_bytes;
 * admitted requests are batched into launches on n_streams streams as they
 * arrive, so work of several batches overlaps on the device. One server per
 * context. Device-resident state kept across requests: planned tool tables
 * (edge points, phase table, group bounds) cached by every input they depend
 * on -- the tool, ap, lead, tilt, step angle, start phase, spindle sense and
 * surface kind (plus fz for round inserts) -- in up to 1/16 of the budget
 * (at most 1 GiB), evicted least recently used first, so a repeated tool and
 * set-up skips the table build; freed device memory stays in the
 * stream-ordered pool for the next admissions; finished maps stay on the
 * device until released. */
fsm_status fsm_server_start(fsm_ctx* ctx, size_t budget_bytes, int32_t n_streams,
                            int32_t max_batch);
fsm_status fsm_server_stop(fsm_ctx* ctx);

/* Queue one prediction (+ roughness). The tool and process are copied.
 * *ticket identifies the request for fsm_poll. Requests larger than the
 * budget fail with FSM_E_NOMEM. */
fsm_status fsm_submit(fsm_ctx* ctx, const fsm_tool* tool, const fsm_process* proc,
                      uint64_t* ticket);

/* Result of a served request. heights is a library-owned device buffer valid
 * until fsm_release_result; rough is a host copy. Latencies in seconds from
 * submission. */
typedef struct {
    void* d_heights;
    int32_t precision, nx, ny, status;
    fsm_roughness_out rough;
    double queue_s, latency_s;
} fsm_result;

/* Wait up to timeout_ms (0 = just check, <0 = forever) for a request.
 * Returns FSM_OK with *out filled, FSM_PENDING (timeout_ms == 0),
 * FSM_E_TIMEOUT (still running after timeout_ms > 0; the request carries
 * on), FSM_E_CANCELLED (see fsm_cancel), or the request's failure status
 * (e.g. FSM_E_NOMEM when its batch could not get device memory). */
fsm_status fsm_poll(fsm_ctx* ctx, uint64_t ticket, int32_t timeout_ms, fsm_result* out);

/* Cancel a request. A request still waiting for admission is removed and
 * never reaches the device; one already admitted finishes its batch (kernels
 * in flight are not interrupted) and its map is freed at completion. Either
 * way fsm_poll then returns FSM_E_CANCELLED and fsm_release_result forgets
 * the ticket. FSM_E_STATE if the request had already finished. */
fsm_status fsm_cancel(fsm_ctx* ctx, uint64_t ticket);

/* Return a finished (or cancelled) request's device memory to the admission
 * budget and forget its ticket. */
fsm_status fsm_release_result(fsm_ctx* ctx, uint64_t ticket);

/* Counters of a running server (no counterpart in the paper). */
typedef struct {
    uint64_t submitted, completed, cancelled, failed, batches;
    uint64_t table_hits, table_misses;   /* requests that found / did not find cached tables */
    uint64_t bytes_in_use, bytes_peak;   /* admission budget in use (maps, tables, scratch) */
    uint64_t table_bytes;                /* of which cached tables */
    int32_t queue_depth, queue_peak;     /* requests waiting for admission */
    int32_t tables_cached, reserved;
} fsm_server_info;
fsm_status fsm_server_stats(fsm_ctx* ctx, fsm_server_info* out);

/* Device-time interval of one served batch: recorded by CUDA events on its
 * slot's stream just before its first kernel and just after its roughness
 * copy, in ms from an origin taken when the server started. Intervals of two
 * slots that intersect show their batches were on the device at the same
 * time. */
typedef struct {
    int32_t slot, n_requests;
    double t_start_ms, t_end_ms;
} fsm_batch_interval;

/* Copy the most recent min(capacity, kept) completed batches (oldest first;
 * the server keeps the last 4096) into out; *n = number copied. */
fsm_status fsm_server_batches(fsm_ctx* ctx, fsm_batch_interval* out, int32_t capacity, int32_t* n);

/* Fault injection for testing the server's failure path (host side only: no
 * device fault is involved): the next `count` device allocations of request
 * height maps report failure without calling the allocator. The batch that
 * contains such a request fails as a whole -- its requests end with
 * FSM_E_NOMEM, their memory goes back to the budget -- and the server keeps
 * serving later requests. count = 0 clears it. */
fsm_status fsm_server_inject_alloc_failures(fsm_ctx* ctx, int32_t count);

#ifdef __cplusplus
}
#endif
#endif
