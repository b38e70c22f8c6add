/*
 * fsm_oracle.h -- plain, slow FP64 CPU oracle of the forward solution method
 * (FSM) for milled-surface topography.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no source, header, table or helper with
 * the CUDA path.
 *
 * What it computes (paper section "Conventional surface topography model"):
 *   - edge points of every tooth (Eq. eq_point_p_equation generalised to
 *     tabulated flat / ball end-mill profiles, with helix lag and axis runout),
 *   - the kinematic chain of Eq. eq_full_transformation,
 *        w = T_SW * T_A * T_TS * T_CT * P_C,
 *     built from 4x4 homogeneous matrices (T_A = lead/tilt orientation is an
 *     extension; the paper's face mill has a vertical axis),
 *   - binning by the sampling boundaries of Eq. eq_sampling_boundaries
 *     (half-open cells) and the per-cell minimum of Section 2.3,
 *   - the trajectory map of Section 3.1 (lowest point of each cutting edge
 *     at each time step, with its global coordinates),
 *   - (extension) the side-wall surface: the same points binned on the
 *     plane of a wall instead of the floor,
 *   - (extension) the ISO Gaussian S- and L-filters that the paper applies
 *     to its measured surfaces (Section 4.1.1), for comparing predictions,
 *   - the areal (Sa, Sq, Sp, Sv, Sz, Ssk, Sku) and line (Ra, Rz) roughness
 *     indicators named in Section 4.1.2 (ISO 25178-2 / ISO 4287 definitions;
 *     the paper gives no formulas).
 *
 * Loops run in the paper's order: time step -> tooth -> edge point.
 * Parity pins: see tests/test_oracle_pins.py. The roughness of the paper's
 * own predicted surfaces is printed only in figures, so agreement with the
 * paper's numerical results is "parity unpinned"; every other function here
 * is pinned by closed forms, invariants or brute force.
 */
#ifndef FSM_ORACLE_H
#define FSM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_TEETH 16

enum { ORC_FLAT = 0, ORC_BALL = 1, ORC_INSERT = 2, ORC_TORUS = 3 };

/* Cutting tool. Angles in degrees, lengths in mm. */
typedef struct {
    int32_t kind;          /* ORC_FLAT, ORC_BALL, ORC_INSERT or ORC_TORUS */
    int32_t n_teeth;       /* 1..ORC_MAX_TEETH */
    int32_t n_edge;        /* flank (flat) or meridian (ball) points, >= 2 */
    int32_t n_end;         /* flat bottom-edge points, 0 or >= 2 (flat, torus; else 0) */
    double diameter;       /* D */
    double helix_deg[ORC_MAX_TEETH];  /* helix angle of each tooth */
    double tooth_deg[ORC_MAX_TEETH];  /* angular position of each tooth */
    double runout_mm;      /* axis offset rho, rotates with the spindle */
    double runout_phase_deg; /* its phase lambda in the rotating frame */
    /* round indexable inserts (ORC_INSERT, Eq. eq_point_p_equation and
     * eq_cutting_edge_to_tool): insert radius R, radial and axial rake, and
     * the per-insert radial/axial runout steps (insert K is offset K*eps) */
    double insert_radius;
    double rake_f_deg, rake_p_deg;
    double eps_r_mm, eps_a_mm;
    /* bull-nose end mill (ORC_TORUS, an extension): corner radius rc,
     * 0 < rc <= D/2; n_end bottom points on the flat part, n_edge points
     * along the corner arc and the flank */
    double corner_radius;
} orc_tool;

/* Process and workpiece grid. */
typedef struct {
    double fz;             /* feed per tooth (mm) */
    double rot_step_deg;   /* spindle angle per time step, 360/step integer */
    double phase0_deg;     /* spindle angle at step 0 */
    int32_t rot_sense;     /* +1 or -1 */
    int32_t n_passes;
    double ap;             /* axial depth of cut */
    double lead_deg;       /* axis leans toward +X (feed) */
    double tilt_deg;       /* axis leans toward +Y (step-over) */
    double ae;             /* step-over between passes (+Y) */
    double pass_x0;        /* tool reference x at the first step of a pass */
    double pass_y0;        /* tool reference y of pass 0 */
    int64_t steps_per_pass;
    double stock_z;        /* un-machined surface height */
    double x0, y0, pitch;  /* grid origin (cell corner) and sampling interval */
    int32_t nx, ny;        /* cells along X (columns) and Y (rows) */
    double z_ref_override; /* NaN: derive from the geometry (see orc_z_ref) */
    /* which surface the map samples: ORC_FLOOR, the horizontal surface
     * (grid over x, y; height z), or ORC_WALL, the side wall that the flank
     * leaves on the +Y side of a single pass (grid over x and z, height
     * along the wall's outward normal -Y, i.e. -y; un-machined at y = wall_y).
     * The tool reference height is the same in both (orc_z_ref). */
    int32_t surface;
    double wall_y;
    /* ORC_ONE_WAY: every pass runs along +X from pass_x0; ORC_ZIGZAG: odd
     * passes run back along -X over the same stretch (step n of an odd pass
     * is where step steps_per_pass-1-n of an even pass is) */
    int32_t pass_mode;
    /* (extension; the paper feeds along one axis) direction of the feed in
     * the XY plane, degrees counter-clockwise from +X: the whole tool path
     * and tool of the feed_dir_deg = 0 process, orientation included, turned
     * by this angle about the vertical through (pass_x0, pass_y0). Passes
     * then run along (cos, sin) and step over along (-sin, cos). Floors
     * only (0 for a wall). */
    double feed_dir_deg;
} orc_process;

enum { ORC_ONE_WAY = 0, ORC_ZIGZAG = 1 };

enum { ORC_FLOOR = 0, ORC_WALL = 1 };

typedef struct {
    int64_t trajectory_points; /* all (step, tooth, edge point) triples */
    int64_t landed;            /* points whose (x,y) falls inside the grid */
    int64_t cutting;           /* landed points with z < stock_z */
    int64_t cells_hit;         /* cells that received >= 1 landed point */
    int64_t cells_flagged;     /* cells next to a boundary-tie point */
    double z_ref;              /* tool reference height used */
} orc_stats;

#define ORC_MAX_PROFILES 16

typedef struct {
    double n, mean, zmin, zmax;
    double Sa, Sq, Sp, Sv, Sz, Ssk, Sku;
    int32_t n_rows, n_cols;
    int32_t row_index[ORC_MAX_PROFILES], col_index[ORC_MAX_PROFILES];
    double Ra_row[ORC_MAX_PROFILES], Rz_row[ORC_MAX_PROFILES];
    double Ra_col[ORC_MAX_PROFILES], Rz_col[ORC_MAX_PROFILES];
} orc_rough;

/* Number of edge points per tooth at a given refinement (1 = as described). */
int orc_points_per_tooth(const orc_tool* t, int refine);

/* Tool-frame edge points P_T = T_CT * P_C (x, y, z per point, tooth-major),
 * at refinement `refine`. Returns the count written, or -1 on bad input. */
int orc_edge_points(const orc_tool* t, const orc_process* p, int refine,
                    double* xyz, int capacity);

/* Height of the tool reference point: the lowest position any edge point
 * reaches during a revolution sits at stock_z - ap. */
double orc_z_ref(const orc_tool* t, const orc_process* p, int refine);

/* Workpiece-frame position of edge point j of tooth K at global step s. */
int orc_pose(const orc_tool* t, const orc_process* p, int64_t s, int K, int j,
             double w[3]);

/* The FSM: scatter every trajectory point into the height map H[ny][nx]
 * (row-major, initialised to stock_z) keeping the minimum z per cell.
 * flags (may be NULL) marks cells next to a point within 1e-12 mm of a
 * sampling boundary. n_threads > 1 splits the global time steps into
 * n_threads contiguous ranges, each swept by one thread into a private map;
 * the maps are merged by min (exact: the per-cell minimum does not depend on
 * the order of the points), hit and tie marks by union, counts by sum.
 * Returns 0 or -1. */
int orc_fsm(const orc_tool* t, const orc_process* p, double* H,
            uint8_t* flags, orc_stats* st, int n_threads);

/* Brute-force inverse: for every cell of the window [i0,i0+ni) x [k0,k0+nk),
 * the minimum z over all trajectory points of the `refine`-times denser
 * sample set (time and edge) that fall inside that cell's sampling
 * boundaries, tested in the centre +- pitch/2 form. Hw[nk][ni]. */
int orc_gather(const orc_tool* t, const orc_process* p, int refine,
               int i0, int k0, int ni, int nk, double* Hw);

/* Trajectory map: for the global time steps s0 .. s0+count-1 (s = pass *
 * steps_per_pass + local step) and every tooth K, the edge point of lowest
 * map height (workpiece z on the floor, -y on a wall; the first in edge
 * order among equal heights) and its map-frame coordinates (floor: x, y, z;
 * wall: x, z, -y):
 * xyz[((s-s0)*n_teeth + K)*3 + d], jmin[(s-s0)*n_teeth + K]. Returns 0 or -1. */
int orc_trajectory(const orc_tool* t, const orc_process* p, int64_t s0, int64_t count,
                   double* xyz, int32_t* jmin);

/* Areal and profile roughness of H[ny][nx]. */
int orc_roughness(const double* H, int nx, int ny, int n_rows, int n_cols,
                  orc_rough* out);

/* Areal Gaussian filtering (ISO 16610-61 weighting function; the paper's
 * measurements use an S-filter of 10 um and an L-filter of 0.8 mm, Section
 * 4.1.1). Weighting function s(x) = exp(-pi (x / (alpha lambda))^2) / (alpha
 * lambda), alpha = sqrt(ln 2 / pi), sampled at the cells t * pitch for
 * |t| <= T = floor(lambda / pitch) (truncated at +-lambda) and applied with
 * the zero-order end correction: each output divides by the sum of the
 * weights that fall inside the map (ISO 16610-28). Rows (x) then columns (y);
 * for a rectangle this equals the 2D weighting function (it is separable).
 *   orc_gauss_filter: out = G_lambda * H (lambda > 0).
 *   orc_sl_surface:   S = G_ls * H (H itself if lambda_s == 0), then
 *                     out = S - G_lc * S (S itself if lambda_c == 0).
 * out may not alias H. Returns 0 or -1. */
int orc_gauss_filter(const double* H, int nx, int ny, double pitch, double lambda, double* out);
int orc_sl_surface(const double* H, int nx, int ny, double pitch, double lambda_s, double lambda_c,
                   double* out);

#ifdef __cplusplus
}
#endif
#endif
