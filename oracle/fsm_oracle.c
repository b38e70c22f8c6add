/*
 * fsm_oracle.c -- plain FP64 CPU oracle of the FSM surface generator.
 *
 * TEST INFRASTRUCTURE ONLY (see fsm_oracle.h). Written for readability
 * against the paper, not for speed: 4x4 homogeneous matrices, loops in the
 * order time step -> tooth -> edge point, one conditional minimum per point.
 */
#define _DEFAULT_SOURCE
#include "fsm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define DEG (M_PI / 180.0)
#define TIE_MM 1e-12 /* a point this close to a sampling boundary is a tie */

/* ------------------------------------------------------------------ */
/* 4x4 homogeneous matrices (Section 3.2: "fixed-size 4x4 matrices").  */
/* ------------------------------------------------------------------ */
typedef struct { double a[4][4]; } mat4;

static mat4 m_identity(void) {
    mat4 m;
    memset(&m, 0, sizeof m);
    for (int i = 0; i < 4; ++i) m.a[i][i] = 1.0;
    return m;
}

static mat4 m_mul(mat4 x, mat4 y) {
    mat4 r;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) acc += x.a[i][k] * y.a[k][j];
            r.a[i][j] = acc;
        }
    return r;
}

static void m_apply(const mat4* m, const double p[3], double out[3]) {
    for (int i = 0; i < 3; ++i)
        out[i] = m->a[i][0] * p[0] + m->a[i][1] * p[1] + m->a[i][2] * p[2] + m->a[i][3];
}

static mat4 m_translate(double x, double y, double z) {
    mat4 m = m_identity();
    m.a[0][3] = x;
    m.a[1][3] = y;
    m.a[2][3] = z;
    return m;
}

/* Rotation about Z by +ang (counter-clockwise seen from +Z). */
static mat4 m_rot_z(double ang) {
    mat4 m = m_identity();
    m.a[0][0] = cos(ang); m.a[0][1] = -sin(ang);
    m.a[1][0] = sin(ang); m.a[1][1] = cos(ang);
    return m;
}

static mat4 m_rot_x(double ang) {
    mat4 m = m_identity();
    m.a[1][1] = cos(ang); m.a[1][2] = -sin(ang);
    m.a[2][1] = sin(ang); m.a[2][2] = cos(ang);
    return m;
}

static mat4 m_rot_y(double ang) {
    mat4 m = m_identity();
    m.a[0][0] = cos(ang);  m.a[0][2] = sin(ang);
    m.a[2][0] = -sin(ang); m.a[2][2] = cos(ang);
    return m;
}

/* T_TS of Eq. eq_tool_to_spindle: [[cos a, sin a], [-sin a, cos a]] with
 * a = phi + 2 pi (K-1)/z_n - omega t. The tooth term lives in T_CT below, so
 * here a = -theta where theta is the spindle angle of the time step. */
static mat4 m_tool_to_spindle(double theta) {
    double a = -theta;
    mat4 m = m_identity();
    m.a[0][0] = cos(a);  m.a[0][1] = sin(a);
    m.a[1][0] = -sin(a); m.a[1][1] = cos(a);
    return m;
}

/* Orientation of the tool axis: lead leans it toward +X, tilt toward +Y. */
static mat4 m_orientation(const orc_process* p) {
    return m_mul(m_rot_x(-p->tilt_deg * DEG), m_rot_y(p->lead_deg * DEG));
}

/* ------------------------------------------------------------------ */
/* Validation and discretisation (Section 2.2).                        */
/* ------------------------------------------------------------------ */
static int64_t steps_per_rev(const orc_process* p) {
    if (!(p->rot_step_deg > 0.0)) return -1;
    double r = 360.0 / p->rot_step_deg;
    int64_t S = (int64_t)llround(r);
    if (S < 1 || fabs(r - (double)S) > 1e-9 * (double)S) return -1;
    return S;
}

static int valid(const orc_tool* t, const orc_process* p) {
    if (!t || !p) return 0;
    if (t->kind != ORC_FLAT && t->kind != ORC_BALL && t->kind != ORC_INSERT && t->kind != ORC_TORUS) return 0;
    if (t->kind == ORC_INSERT && !(t->insert_radius > 0.0)) return 0;
    if (t->kind == ORC_TORUS && !(t->corner_radius > 0.0 && t->corner_radius <= 0.5 * t->diameter)) return 0;
    if (t->n_teeth < 1 || t->n_teeth > ORC_MAX_TEETH) return 0;
    if (t->n_edge < 2) return 0;
    int has_end = t->kind == ORC_FLAT || t->kind == ORC_TORUS;
    if (has_end && (t->n_end == 1 || t->n_end < 0)) return 0;
    if (!has_end && t->n_end != 0) return 0;
    if (!(t->diameter > 0.0)) return 0;
    if (steps_per_rev(p) < 0) return 0;
    if (!(p->fz > 0.0) || !(p->ap > 0.0) || !(p->pitch > 0.0)) return 0;
    if (p->rot_sense != 1 && p->rot_sense != -1) return 0;
    if (p->n_passes < 1 || p->steps_per_pass < 1) return 0;
    if (p->nx < 1 || p->ny < 1) return 0;
    if (p->surface != ORC_FLOOR && p->surface != ORC_WALL) return 0;
    if (p->surface == ORC_WALL && p->n_passes != 1) return 0;
    if (p->pass_mode != ORC_ONE_WAY && p->pass_mode != ORC_ZIGZAG) return 0;
    if (!isfinite(p->feed_dir_deg)) return 0;
    if (p->surface == ORC_WALL && p->feed_dir_deg != 0.0) return 0;
    return 1;
}

/* Workpiece point -> map frame: the floor keeps (x, y, z); a wall on the +Y
 * side is sampled over (x, z) with height -y (outward normal -Y). */
static void to_map_frame(const orc_process* p, const double w[3], double out[3]) {
    if (p->surface == ORC_WALL) {
        double x = w[0], y = w[1], z = w[2];
        out[0] = x;
        out[1] = z;
        out[2] = -y;
    } else {
        out[0] = w[0];
        out[1] = w[1];
        out[2] = w[2];
    }
}

/* Height of the un-machined surface in the map frame. */
static double map_stock(const orc_process* p) {
    return p->surface == ORC_WALL ? -p->wall_y : p->stock_z;
}

int orc_points_per_tooth(const orc_tool* t, int refine) {
    if (!t || refine < 1 || t->n_edge < 2) return -1;
    int edge = (t->n_edge - 1) * refine + 1;
    int end = ((t->kind == ORC_FLAT || t->kind == ORC_TORUS) && t->n_end >= 2) ? (t->n_end - 1) * refine + 1 : 0;
    return edge + end;
}

/* Round insert (Section 2.2, Eq. eq_tool_point_p_equation): N points with
 * l uniform in [-dL, dL], dL = max(sqrt(R^2 - (R - ap)^2), fz / (2 cos g_f)),
 * on the lower semicircle z = R - sqrt(R^2 - l^2) (cutting-edge frame, origin
 * at the insert's lowest point). dL is capped at R (the semicircle's end). */
static void insert_point(const orc_tool* t, const orc_process* p, int refine, int j, double* l, double* z) {
    double R = t->insert_radius;
    int edge = (t->n_edge - 1) * refine + 1;
    double imm = R - p->ap;
    double dl_ap = p->ap >= R ? R : sqrt(R * R - imm * imm);
    double dl_fz = p->fz / (2.0 * cos(t->rake_f_deg * DEG));
    double dL = dl_ap > dl_fz ? dl_ap : dl_fz;
    if (dL > R) dL = R;
    *l = -dL + 2.0 * dL * ((double)j / (double)(edge - 1));
    *z = R - sqrt(R * R - (*l) * (*l));
}

/* Radius and height (in the tool frame, origin at the tool tip on the axis)
 * of edge point j of the profile. Flat end: bottom edge first (h = 0, r from
 * 0 to D/2), then the flank (r = D/2, h from 0 to ap). Ball end: points
 * uniform in polar angle kappa on the sphere of radius D/2, over the cap
 * that can reach below the stock for the given lead/tilt. */
static void profile_point(const orc_tool* t, const orc_process* p, int refine,
                          int j, double* r, double* h) {
    double R = 0.5 * t->diameter;
    int edge = (t->n_edge - 1) * refine + 1;
    if (t->kind == ORC_FLAT) {
        int end = t->n_end >= 2 ? (t->n_end - 1) * refine + 1 : 0;
        if (j < end) {
            *r = R * ((double)j / (double)(end - 1));
            *h = 0.0;
        } else {
            int f = j - end;
            *r = R;
            *h = p->ap * ((double)f / (double)(edge - 1));
        }
        return;
    }
    if (t->kind == ORC_TORUS) {
        /* bottom flat r in [0, R - rc] at h = 0, then points uniform in arc
         * length along the corner arc (centre (R - rc, rc)) and the flank,
         * from the bottom up to height ap */
        double rc = t->corner_radius;
        int end = t->n_end >= 2 ? (t->n_end - 1) * refine + 1 : 0;
        if (j < end) {
            *r = (R - rc) * ((double)j / (double)(end - 1));
            *h = 0.0;
            return;
        }
        double arc_top = p->ap >= rc ? 0.5 * M_PI : acos(1.0 - p->ap / rc);
        double len_arc = rc * arc_top;
        double len = len_arc + (p->ap > rc ? p->ap - rc : 0.0);
        double s_along = len * ((double)(j - end) / (double)(edge - 1));
        if (s_along <= len_arc) {
            double kappa = s_along / rc;
            *r = R - rc + rc * sin(kappa);
            *h = rc * (1.0 - cos(kappa));
        } else {
            *r = R;
            *h = rc + (s_along - len_arc);
        }
        return;
    }
    double a22 = cos(p->tilt_deg * DEG) * cos(p->lead_deg * DEG);
    if (a22 > 1.0) a22 = 1.0;
    double tau = acos(a22);
    double c = (R - p->ap) / R;
    if (c < -1.0) c = -1.0;
    if (c > 1.0) c = 1.0;
    double half = acos(c);
    double klo = tau - half > 0.0 ? tau - half : 0.0;
    double khi = tau + half < 0.5 * M_PI ? tau + half : 0.5 * M_PI;
    double kappa = klo + (khi - klo) * ((double)j / (double)(edge - 1));
    *r = R * sin(kappa);
    *h = R * (1.0 - cos(kappa));
}

/* T_CT for an end mill: place the profile point at the tooth's angular
 * position, lagged by the helix (psi = h tan(beta) / (D/2)), and offset by
 * the axis runout that rotates with the spindle. */
/* T_CT of Eq. eq_cutting_edge_to_tool for insert K (0-based, so the
 * paper's K-1 is K here): rake rotation and the translation
 * (D/2 + K eps_r, 0, K eps_a). */
static mat4 m_insert_to_tool(const orc_tool* t, int K) {
    double gf = t->rake_f_deg * DEG, gp = t->rake_p_deg * DEG;
    mat4 m = m_identity();
    m.a[0][0] = cos(gf);  m.a[0][1] = sin(gf) * cos(gp); m.a[0][2] = sin(gf) * sin(gp);
    m.a[1][0] = -sin(gf); m.a[1][1] = cos(gf) * cos(gp); m.a[1][2] = cos(gf) * sin(gp);
    m.a[2][0] = 0.0;      m.a[2][1] = -sin(gp);          m.a[2][2] = cos(gp);
    m.a[0][3] = 0.5 * t->diameter + (double)K * t->eps_r_mm;
    m.a[1][3] = 0.0;
    m.a[2][3] = (double)K * t->eps_a_mm;
    return m;
}

static void tool_point(const orc_tool* t, const orc_process* p, int refine,
                       int K, int j, double out[3]) {
    if (t->kind == ORC_INSERT) {
        /* insert K sits at -tooth_deg[K] about the axis (the 2 pi (K-1)/z_n
         * of Eq. eq_tool_to_spindle), then the spindle-axis runout */
        double l, z;
        insert_point(t, p, refine, j, &l, &z);
        double lam = t->runout_phase_deg * DEG;
        mat4 m = m_mul(m_mul(m_translate(t->runout_mm * cos(lam), t->runout_mm * sin(lam), 0.0),
                             m_rot_z(-t->tooth_deg[K] * DEG)),
                       m_insert_to_tool(t, K));
        double pc[3] = {l, 0.0, z};
        m_apply(&m, pc, out);
        return;
    }
    double r, h;
    profile_point(t, p, refine, j, &r, &h);
    double psi = h * tan(t->helix_deg[K] * DEG) / (0.5 * t->diameter);
    double alpha = -t->tooth_deg[K] * DEG - (double)p->rot_sense * psi;
    double lam = t->runout_phase_deg * DEG;
    mat4 tct = m_mul(m_translate(t->runout_mm * cos(lam), t->runout_mm * sin(lam), 0.0),
                     m_rot_z(alpha));
    double pc[3] = {r, 0.0, h};
    m_apply(&tct, pc, out);
}

int orc_edge_points(const orc_tool* t, const orc_process* p, int refine,
                    double* xyz, int capacity) {
    if (!valid(t, p) || refine < 1) return -1;
    int E = orc_points_per_tooth(t, refine);
    int total = E * t->n_teeth;
    if (capacity < total) return -1;
    for (int K = 0; K < t->n_teeth; ++K)
        for (int j = 0; j < E; ++j) tool_point(t, p, refine, K, j, xyz + 3 * (K * E + j));
    return total;
}

double orc_z_ref(const orc_tool* t, const orc_process* p, int refine) {
    if (!valid(t, p) || refine < 1) return NAN;
    mat4 A = m_orientation(p);
    double a2xy = sqrt(A.a[2][0] * A.a[2][0] + A.a[2][1] * A.a[2][1]);
    int E = orc_points_per_tooth(t, refine);
    double lowest = INFINITY;
    for (int K = 0; K < t->n_teeth; ++K)
        for (int j = 0; j < E; ++j) {
            double q[3];
            tool_point(t, p, refine, K, j, q);
            /* lowest z of this point over one spin about the tool axis */
            double zlow = A.a[2][2] * q[2] - a2xy * sqrt(q[0] * q[0] + q[1] * q[1]);
            if (zlow < lowest) lowest = zlow;
        }
    return p->stock_z - p->ap - lowest;
}

static double resolved_z_ref(const orc_tool* t, const orc_process* p) {
    return isnan(p->z_ref_override) ? orc_z_ref(t, p, 1) : p->z_ref_override;
}

/* T_SW * T_A * T_TS for pass `pass`, local step n expressed as
 * nq + nr/refine, with the global spindle step split the same way. */
static mat4 step_matrix(const orc_tool* t, const orc_process* p, const mat4* A,
                        double z_ref, int refine, int pass, int64_t nq, int64_t nr) {
    int64_t S = steps_per_rev(p);
    double fs = (double)t->n_teeth * p->fz / (double)S; /* feed per time step */
    int64_t sq = (int64_t)pass * p->steps_per_pass + nq; /* whole steps */
    int64_t m = sq % S;                                  /* spindle phase */
    double theta = (p->phase0_deg + (double)p->rot_sense *
                    ((double)m * p->rot_step_deg +
                     (double)nr * (p->rot_step_deg / (double)refine))) * DEG;
    double xc;
    if (p->pass_mode == ORC_ZIGZAG && (pass & 1)) /* run back: step n sits at step spp-1-n */
        xc = p->pass_x0 + ((double)(p->steps_per_pass - 1 - nq) * fs - (double)nr * (fs / (double)refine));
    else
        xc = p->pass_x0 + ((double)nq * fs + (double)nr * (fs / (double)refine));
    double yc = p->pass_y0 + (double)pass * p->ae;
    mat4 tsw = m_translate(xc, yc, z_ref);
    mat4 tts = m_tool_to_spindle(theta);
    mat4 T = m_mul(m_mul(tsw, *A), tts);
    if (p->feed_dir_deg != 0.0) {
        /* feed direction: the chain above, turned about the vertical through
         * the start of pass 0 */
        mat4 F = m_mul(m_mul(m_translate(p->pass_x0, p->pass_y0, 0.0), m_rot_z(p->feed_dir_deg * DEG)),
                       m_translate(-p->pass_x0, -p->pass_y0, 0.0));
        T = m_mul(F, T);
    }
    return T;
}

int orc_pose(const orc_tool* t, const orc_process* p, int64_t s, int K, int j,
             double w[3]) {
    if (!valid(t, p) || s < 0 || K < 0 || K >= t->n_teeth) return -1;
    int E = orc_points_per_tooth(t, 1);
    if (j < 0 || j >= E) return -1;
    int pass = (int)(s / p->steps_per_pass);
    int64_t n = s % p->steps_per_pass;
    mat4 A = m_orientation(p);
    mat4 T = step_matrix(t, p, &A, resolved_z_ref(t, p), 1, pass, n, 0);
    double q[3];
    tool_point(t, p, 1, K, j, q);
    m_apply(&T, q, w);
    return 0;
}

/* ------------------------------------------------------------------ */
/* The FSM scatter (Section 2.3, flowchart FSM_Flowchart).             */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_tool* t;
    const orc_process* p;
    int64_t s_begin, s_end;  /* global time steps [s_begin, s_end) of this thread */
    double z_ref;
    double* H;
    uint8_t* flags;
    uint8_t* hit;
    orc_stats st;
} fsm_job;

static void flag_point(const orc_process* p, double wx, double wy, uint8_t* flags) {
    double fx = (wx - p->x0) / p->pitch, fy = (wy - p->y0) / p->pitch;
    long ix[2], iy[2];
    int nxs = 1, nys = 1;
    ix[0] = (long)floor(fx);
    iy[0] = (long)floor(fy);
    long bx = lround(fx), by = lround(fy);
    int tie_x = fabs(wx - (p->x0 + (double)bx * p->pitch)) < TIE_MM;
    int tie_y = fabs(wy - (p->y0 + (double)by * p->pitch)) < TIE_MM;
    if (!tie_x && !tie_y) return;
    if (tie_x) { ix[0] = bx - 1; ix[1] = bx; nxs = 2; }
    if (tie_y) { iy[0] = by - 1; iy[1] = by; nys = 2; }
    for (int a = 0; a < nys; ++a)
        for (int b = 0; b < nxs; ++b)
            if (iy[a] >= 0 && iy[a] < p->ny && ix[b] >= 0 && ix[b] < p->nx)
                flags[(size_t)iy[a] * p->nx + ix[b]] = 1;
}

static void* fsm_worker(void* arg) {
    fsm_job* job = (fsm_job*)arg;
    const orc_tool* t = job->t;
    const orc_process* p = job->p;
    int E = orc_points_per_tooth(t, 1);
    int N = t->n_teeth;
    double* q = (double*)malloc(sizeof(double) * 3 * (size_t)E * N);
    for (int K = 0; K < N; ++K)
        for (int j = 0; j < E; ++j) tool_point(t, p, 1, K, j, q + 3 * (K * E + j));
    mat4 A = m_orientation(p);
    const double stock = map_stock(p);
    for (int64_t s = job->s_begin; s < job->s_end; ++s) {          /* time step */
        int pass = (int)(s / p->steps_per_pass);
        int64_t n = s - (int64_t)pass * p->steps_per_pass;
        mat4 T = step_matrix(t, p, &A, job->z_ref, 1, pass, n, 0);
        for (int K = 0; K < N; ++K) {                               /* tooth */
            for (int j = 0; j < E; ++j) {                           /* edge point */
                double wp[3], w[3];
                m_apply(&T, q + 3 * (K * E + j), wp);
                to_map_frame(p, wp, w);
                job->st.trajectory_points++;
                double cx = floor((w[0] - p->x0) / p->pitch);
                double cy = floor((w[1] - p->y0) / p->pitch);
                int inside = cx >= 0.0 && cx < (double)p->nx && cy >= 0.0 && cy < (double)p->ny;
                if (w[2] < stock && job->flags) flag_point(p, w[0], w[1], job->flags);
                if (!inside) continue;
                size_t cell = (size_t)cy * p->nx + (size_t)cx;
                job->st.landed++;
                job->hit[cell] = 1;
                if (w[2] < stock) job->st.cutting++;
                if (w[2] < job->H[cell]) job->H[cell] = w[2]; /* keep the lowest z */
            }
        }
    }
    free(q);
    return NULL;
}

/* Merge of the threads' private maps over the cells [c_begin, c_end): the
 * per-cell minimum is order-free, so the merged map is the single-thread
 * map exactly; hit and boundary-tie marks are unions. */
typedef struct {
    fsm_job* jobs;
    int n_threads;
    size_t c_begin, c_end;
} merge_job;

static void* merge_worker(void* arg) {
    merge_job* m = (merge_job*)arg;
    fsm_job* j0 = &m->jobs[0];
    for (int i = 1; i < m->n_threads; ++i) {
        const fsm_job* ji = &m->jobs[i];
        for (size_t c = m->c_begin; c < m->c_end; ++c) {
            if (ji->H[c] < j0->H[c]) j0->H[c] = ji->H[c];
            j0->hit[c] |= ji->hit[c];
            if (j0->flags) j0->flags[c] |= ji->flags[c];
        }
    }
    return NULL;
}

/* Contiguous share [lo, hi) of `total` items for part i of n. */
static void share(int64_t total, int i, int n, int64_t* lo, int64_t* hi) {
    *lo = total / n * i + (i < total % n ? i : total % n);
    *hi = *lo + total / n + (i < total % n ? 1 : 0);
}

int orc_fsm(const orc_tool* t, const orc_process* p, double* H, uint8_t* flags,
            orc_stats* st, int n_threads) {
    if (!valid(t, p) || !H) return -1;
    const int64_t steps = (int64_t)p->n_passes * p->steps_per_pass;
    if (n_threads < 1) n_threads = 1;
    if ((int64_t)n_threads > steps) n_threads = (int)steps;
    size_t cells = (size_t)p->nx * (size_t)p->ny;
    double z_ref = resolved_z_ref(t, p);
    fsm_job* jobs = (fsm_job*)calloc((size_t)n_threads, sizeof(fsm_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int i = 0; i < n_threads; ++i) {
        jobs[i].t = t;
        jobs[i].p = p;
        share(steps, i, n_threads, &jobs[i].s_begin, &jobs[i].s_end);
        jobs[i].z_ref = z_ref;
        jobs[i].H = (i == 0) ? H : (double*)malloc(sizeof(double) * cells);
        jobs[i].flags = flags ? (i == 0 ? flags : (uint8_t*)calloc(cells, 1)) : NULL;
        jobs[i].hit = (uint8_t*)calloc(cells, 1);
        for (size_t c = 0; c < cells; ++c) jobs[i].H[c] = map_stock(p);
        if (i == 0 && flags) memset(flags, 0, cells);
    }
    for (int i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, fsm_worker, &jobs[i]);
    fsm_worker(&jobs[0]);
    for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    if (n_threads > 1) {
        merge_job* mj = (merge_job*)calloc((size_t)n_threads, sizeof(merge_job));
        for (int i = 0; i < n_threads; ++i) {
            int64_t lo, hi;
            share((int64_t)cells, i, n_threads, &lo, &hi);
            mj[i].jobs = jobs;
            mj[i].n_threads = n_threads;
            mj[i].c_begin = (size_t)lo;
            mj[i].c_end = (size_t)hi;
        }
        for (int i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, merge_worker, &mj[i]);
        merge_worker(&mj[0]);
        for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
        free(mj);
    }
    orc_stats total;
    memset(&total, 0, sizeof total);
    for (int i = 0; i < n_threads; ++i) {
        if (i > 0) {
            free(jobs[i].H);
            if (flags) free(jobs[i].flags);
        }
        total.trajectory_points += jobs[i].st.trajectory_points;
        total.landed += jobs[i].st.landed;
        total.cutting += jobs[i].st.cutting;
    }
    for (size_t c = 0; c < cells; ++c) {
        total.cells_hit += jobs[0].hit[c];
        if (flags) total.cells_flagged += flags[c];
    }
    total.z_ref = z_ref;
    for (int i = 0; i < n_threads; ++i) free(jobs[i].hit);
    free(jobs);
    free(th);
    if (st) *st = total;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Brute-force inverse: per-cell minimum over a (refined) sample set.  */
/* ------------------------------------------------------------------ */
/* ------------------------------------------------------------------ */
/* Trajectory map (Section 3.1, trajectory computation module): at each */
/* time step, the lowest point of every cutting edge and its global     */
/* coordinates, computed from the same transformed points as the map.   */
/* ------------------------------------------------------------------ */
int orc_trajectory(const orc_tool* t, const orc_process* p, int64_t s0, int64_t count,
                   double* xyz, int32_t* jmin) {
    if (!valid(t, p) || s0 < 0 || count < 0 || !xyz || !jmin) return -1;
    int64_t total = (int64_t)p->n_passes * p->steps_per_pass;
    if (s0 + count > total) return -1;
    int E = orc_points_per_tooth(t, 1);
    int N = t->n_teeth;
    double* q = (double*)malloc(sizeof(double) * 3 * (size_t)E * N);
    for (int K = 0; K < N; ++K)
        for (int j = 0; j < E; ++j) tool_point(t, p, 1, K, j, q + 3 * (K * E + j));
    mat4 A = m_orientation(p);
    double z_ref = resolved_z_ref(t, p);
    for (int64_t s = s0; s < s0 + count; ++s) {                 /* time step */
        int pass = (int)(s / p->steps_per_pass);
        mat4 T = step_matrix(t, p, &A, z_ref, 1, pass, s % p->steps_per_pass, 0);
        for (int K = 0; K < N; ++K) {                           /* cutting edge */
            double best[3] = {0.0, 0.0, INFINITY};
            int32_t bj = -1;
            for (int j = 0; j < E; ++j) {                       /* edge point */
                double wp[3], w[3];
                m_apply(&T, q + 3 * (K * E + j), wp);
                to_map_frame(p, wp, w);
                if (w[2] < best[2]) {  /* strict: the first point in edge order wins a tie */
                    best[0] = w[0]; best[1] = w[1]; best[2] = w[2];
                    bj = j;
                }
            }
            size_t r = (size_t)(s - s0) * N + K;
            xyz[3 * r] = best[0];
            xyz[3 * r + 1] = best[1];
            xyz[3 * r + 2] = best[2];
            jmin[r] = bj;
        }
    }
    free(q);
    return 0;
}

int orc_gather(const orc_tool* t, const orc_process* p, int refine,
               int i0, int k0, int ni, int nk, double* Hw) {
    if (!valid(t, p) || refine < 1 || ni < 1 || nk < 1 || !Hw) return -1;
    int E = orc_points_per_tooth(t, refine);
    int N = t->n_teeth;
    double z_ref = resolved_z_ref(t, p); /* the unrefined tool's reference */
    double* q = (double*)malloc(sizeof(double) * 3 * (size_t)E * N);
    for (int K = 0; K < N; ++K)
        for (int j = 0; j < E; ++j) tool_point(t, p, refine, K, j, q + 3 * (K * E + j));
    mat4 A = m_orientation(p);
    /* every trajectory point of the refined set that lies below the stock
     * and inside the window's outer sampling boundaries */
    double wx_lo = p->x0 + (double)i0 * p->pitch - p->pitch;
    double wx_hi = p->x0 + (double)(i0 + ni) * p->pitch + p->pitch;
    double wy_lo = p->y0 + (double)k0 * p->pitch - p->pitch;
    double wy_hi = p->y0 + (double)(k0 + nk) * p->pitch + p->pitch;
    size_t cap = 1 << 16, np = 0;
    double* pts = (double*)malloc(sizeof(double) * 3 * cap);
    for (int pass = 0; pass < p->n_passes; ++pass) {
        int64_t nsteps = (p->steps_per_pass - 1) * refine + 1;
        for (int64_t n = 0; n < nsteps; ++n) {
            mat4 T = step_matrix(t, p, &A, z_ref, refine, pass, n / refine, n % refine);
            for (int K = 0; K < N; ++K)
                for (int j = 0; j < E; ++j) {
                    double wp[3], w[3];
                    m_apply(&T, q + 3 * (K * E + j), wp);
                    to_map_frame(p, wp, w);
                    if (!(w[2] < map_stock(p))) continue;
                    if (w[0] < wx_lo || w[0] > wx_hi || w[1] < wy_lo || w[1] > wy_hi) continue;
                    if (np == cap) {
                        cap *= 2;
                        pts = (double*)realloc(pts, sizeof(double) * 3 * cap);
                    }
                    memcpy(pts + 3 * np, w, sizeof w);
                    ++np;
                }
        }
    }
    /* per cell: sampling boundaries x_i - d/2 <= x < x_i + d/2 (same in y) */
    double half = 0.5 * p->pitch;
    for (int k = 0; k < nk; ++k) {
        double yc = p->y0 + ((double)(k0 + k) + 0.5) * p->pitch;
        for (int i = 0; i < ni; ++i) {
            double xc = p->x0 + ((double)(i0 + i) + 0.5) * p->pitch;
            double best = map_stock(p);
            for (size_t a = 0; a < np; ++a) {
                const double* w = pts + 3 * a;
                if (xc - half <= w[0] && w[0] < xc + half && yc - half <= w[1] && w[1] < yc + half &&
                    w[2] < best)
                    best = w[2];
            }
            Hw[(size_t)k * ni + i] = best;
        }
    }
    free(pts);
    free(q);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Roughness (Section 4.1.2; ISO 25178-2 areal, ISO 4287 line).        */
/* ------------------------------------------------------------------ */
static void line_roughness(const double* z, size_t stride, int L, double* Ra, double* Rz) {
    double mean = 0.0;
    for (int a = 0; a < L; ++a) mean += z[(size_t)a * stride];
    mean /= (double)L;
    double sa = 0.0;
    for (int a = 0; a < L; ++a) sa += fabs(z[(size_t)a * stride] - mean);
    *Ra = sa / (double)L;
    if (L < 5) {
        *Rz = NAN;
        return;
    }
    double rz = 0.0;
    for (int seg = 0; seg < 5; ++seg) {
        int lo = (int)(((int64_t)seg * L) / 5), hi = (int)(((int64_t)(seg + 1) * L) / 5);
        double mx = -INFINITY, mn = INFINITY;
        for (int a = lo; a < hi; ++a) {
            double v = z[(size_t)a * stride];
            if (v > mx) mx = v;
            if (v < mn) mn = v;
        }
        rz += mx - mn;
    }
    *Rz = rz / 5.0;
}

int orc_roughness(const double* H, int nx, int ny, int n_rows, int n_cols, orc_rough* out) {
    if (!H || !out || nx < 1 || ny < 1 || n_rows < 0 || n_cols < 0 ||
        n_rows > ORC_MAX_PROFILES || n_cols > ORC_MAX_PROFILES)
        return -1;
    memset(out, 0, sizeof *out);
    size_t n = (size_t)nx * (size_t)ny;
    double sum = 0.0, mn = INFINITY, mx = -INFINITY;
    for (size_t c = 0; c < n; ++c) {
        sum += H[c];
        if (H[c] < mn) mn = H[c];
        if (H[c] > mx) mx = H[c];
    }
    double mu = sum / (double)n;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double d = H[c] - mu;
        s1 += fabs(d);
        s2 += d * d;
        s3 += d * d * d;
        s4 += d * d * d * d;
    }
    out->n = (double)n;
    out->mean = mu;
    out->zmin = mn;
    out->zmax = mx;
    out->Sa = s1 / (double)n;
    out->Sq = sqrt(s2 / (double)n);
    out->Sp = mx - mu;
    out->Sv = mu - mn;
    out->Sz = out->Sp + out->Sv;
    if (out->Sq > 0.0) {
        out->Ssk = (s3 / (double)n) / (out->Sq * out->Sq * out->Sq);
        out->Sku = (s4 / (double)n) / (out->Sq * out->Sq * out->Sq * out->Sq);
    } else {
        out->Ssk = NAN;
        out->Sku = NAN;
    }
    out->n_rows = n_rows;
    out->n_cols = n_cols;
    for (int r = 0; r < n_rows; ++r) {
        int k = (int)(((int64_t)(2 * r + 1) * ny) / (2 * n_rows));
        out->row_index[r] = k;
        line_roughness(H + (size_t)k * nx, 1, nx, &out->Ra_row[r], &out->Rz_row[r]);
    }
    for (int c = 0; c < n_cols; ++c) {
        int i = (int)(((int64_t)(2 * c + 1) * nx) / (2 * n_cols));
        out->col_index[c] = i;
        line_roughness(H + i, (size_t)nx, ny, &out->Ra_col[c], &out->Rz_col[c]);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* ISO 16610-61 areal Gaussian filter (see fsm_oracle.h).              */
/* ------------------------------------------------------------------ */
static int gauss_weights(double pitch, double lambda, double** g_out) {
    int T = (int)floor(lambda / pitch + 1e-9);
    double a = sqrt(log(2.0) / M_PI) * lambda;  /* alpha * lambda */
    double* g = (double*)malloc(sizeof(double) * (size_t)(2 * T + 1));
    for (int t = -T; t <= T; ++t) {
        double x = (double)t * pitch / a;
        g[t + T] = exp(-M_PI * x * x) / a;   /* s(t * pitch) */
    }
    *g_out = g;
    return T;
}

/* one line of n samples with stride `stride`: out[i] = sum_t g[t] in[i+t] /
 * sum_t g[t], t over the weights whose sample lies inside the line */
static void gauss_line(const double* in, double* out, int n, size_t stride, const double* g, int T) {
    for (int i = 0; i < n; ++i) {
        double num = 0.0, den = 0.0;
        for (int t = -T; t <= T; ++t) {
            int j = i + t;
            if (j < 0 || j >= n) continue;
            num += g[t + T] * in[(size_t)j * stride];
            den += g[t + T];
        }
        out[(size_t)i * stride] = num / den;
    }
}

int orc_gauss_filter(const double* H, int nx, int ny, double pitch, double lambda, double* out) {
    if (!H || !out || H == out || nx < 1 || ny < 1 || !(pitch > 0.0) || !(lambda > 0.0)) return -1;
    double* g;
    int T = gauss_weights(pitch, lambda, &g);
    size_t cells = (size_t)nx * (size_t)ny;
    double* tmp = (double*)malloc(sizeof(double) * cells);
    for (int k = 0; k < ny; ++k)   /* rows: along x */
        gauss_line(H + (size_t)k * nx, tmp + (size_t)k * nx, nx, 1, g, T);
    for (int i = 0; i < nx; ++i)   /* columns: along y */
        gauss_line(tmp + i, out + i, ny, (size_t)nx, g, T);
    free(tmp);
    free(g);
    return 0;
}

int orc_sl_surface(const double* H, int nx, int ny, double pitch, double lambda_s, double lambda_c,
                   double* out) {
    if (!H || !out || H == out || nx < 1 || ny < 1 || !(pitch > 0.0) || lambda_s < 0.0 || lambda_c < 0.0)
        return -1;
    size_t cells = (size_t)nx * (size_t)ny;
    double* S = (double*)malloc(sizeof(double) * cells);
    if (lambda_s > 0.0) orc_gauss_filter(H, nx, ny, pitch, lambda_s, S);
    else memcpy(S, H, sizeof(double) * cells);
    if (lambda_c > 0.0) {
        orc_gauss_filter(S, nx, ny, pitch, lambda_c, out);  /* the mean surface */
        for (size_t c = 0; c < cells; ++c) out[c] = S[c] - out[c];
    } else {
        memcpy(out, S, sizeof(double) * cells);
    }
    free(S);
    return 0;
}
