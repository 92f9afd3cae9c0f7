/*
 * mp_oracle.h - CPU oracle for semi-analytical (Pollock 1988) particle
 * tracking on structured grids.  TEST INFRASTRUCTURE ONLY: used by the tests,
 * the smoke check and the benchmark's CPU-baseline leg, never by the product
 * path.  Plain single-threaded IEEE double precision.
 */
#ifndef MP_ORACLE_H
#define MP_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#define ORC_MAX_AXIS 8192
#define ORC_DEFAULT_MAX_STEPS 1000000

/* particle status */
#define ORC_ST_ACTIVE 0
#define ORC_ST_TIME 1
#define ORC_ST_SINK 2
#define ORC_ST_BOUNDARY 3
#define ORC_ST_EXIT_DOMAIN 4
#define ORC_ST_NO_EXIT 5
#define ORC_ST_STEP_CAP 6
#define ORC_ST_INVALID_RELEASE 7

#define ORC_FACE_NONE 255

typedef struct {
    int32_t nlay, nrow, ncol;
    const double* delr;   /* [ncol] */
    const double* delc;   /* [nrow] */
    const double* dz;     /* [nlay] */
    double origin[3];
    const double* qx;     /* [nlay][nrow][ncol+1] */
    const double* qy;     /* [nlay][nrow+1][ncol] */
    const double* qz;     /* [nlay+1][nrow][ncol] */
    const double* porosity; /* [nlay][nrow][ncol] */
    const int8_t* ibound;   /* [nlay][nrow][ncol] */
} orc_field;

typedef struct {
    double t_stop;        /* +inf allowed */
    int32_t n_times;
    const double* times;  /* ascending */
    int64_t max_steps;    /* <= 0: default */
    int32_t pass_weak_sinks; /* 1: enter sink cells, leave through outflow faces */
    int32_t path_start;   /* pathlines: 1 = a record at the start of every particle */
    double weak_sink_fraction; /* > 0 with pass_weak_sinks: a sink cell that
                                  extracts at least this fraction of its
                                  inflow still stops particles */
    int32_t arith;        /* ORC_ARITH_PLAIN (0, the reference) or ORC_ARITH_MIRROR */
    double jitter;        /* > 0: perturb every crossing (tests only, see below) */
    uint64_t jitter_seed;
    int64_t jitter_id0;   /* particle q draws as particle jitter_id0 + q */
} orc_track_opts;

/* Jitter (a test instrument, not part of the method): with jitter = e > 0
 * every completed cell-step's time (which moves the other axes and the clock)
 * is multiplied by (1 + e u1), after the hand-over every transverse offset
 * moves by e u2 D, and a moving particle's start offsets move by e u3 D
 * (clamped to the cell), u1, u2, u3 uniform in [-1, 1) from a counter-based
 * generator (SplitMix64
 * of the seed, the particle's index plus jitter_id0, the step count and the
 * axis).  Runs with
 * e of the order of one FP32 rounding show how far a particle's result moves
 * under perturbations of that size at every step: the spread a
 * reduced-precision evaluation is measured against. */

/* Arithmetic of the in-cell solution.
 * PLAIN (the reference): the method's formulas written out as they read,
 *   vp = v1 + A p, t = (d / vp) (log1p(z) / z) with z = A (d / vp),
 *   p(t) = p + vp t (expm1(w) / w) with w = A t, the C library's log1p and
 *   expm1, IEEE division, no fused multiply-add.
 * MIRROR: the same solution in Pollock's own forms, ln(1 + z) / A and
 *   p + vp (e^{At} - 1) / A, with 1/A formed once per cell, fused
 *   multiply-adds and table-driven log1p / expm1 evaluated by fixed steps,
 *   so that another implementation of the same steps gives the same bits. */
#define ORC_ARITH_PLAIN 0
#define ORC_ARITH_MIRROR 1

/* Rectangular unstructured grid: axis-aligned box cells, per cell and face
 * (x-, x+, y-, y+, z-, z+) a list of sub-faces with the neighbour across
 * (-1: outside), the flow through it (m^3/s along +axis) and its rectangle
 * in the two other axes (lo_a, hi_a, lo_b, hi_b; axes in x, y, z order). */
typedef struct {
    int64_t ncell;
    const double* box;        /* [ncell][6] x0, y0, z0, dx, dy, dz */
    const double* porosity;   /* [ncell] */
    const int8_t* ibound;     /* [ncell] */
    const int64_t* face_off;  /* [6 ncell + 1] */
    const int32_t* nbr;       /* [nsub] */
    const double* q;          /* [nsub] */
    const double* rect;       /* [nsub][4] */
} orc_usg_field;

typedef struct orc_grid orc_grid;

/* One pathline point (Methods, "MODPATH": pathline simulations record the
 * path): the release point and the point reached by every cell-step. */
typedef struct {
    double x, y, z, t;    /* global position (m), time (s) */
    int32_t particle;     /* index in the tracked state */
    int32_t cell;         /* cell the point belongs to after the step */
    uint32_t seq;         /* cell-steps taken since release when the point is reached */
    uint8_t status;       /* status after the step (ACTIVE while moving on) */
    uint8_t pad[3];
} orc_path_rec;

/* One cell-step as the oracle evaluated it: the exit time and the reachable
 * face of every axis, the particle velocity per axis, the time at the start
 * of the step and the axis taken (-1: none). */
typedef struct orc_trace_rec {
    double te[3];         /* exit time per axis (+inf: no reachable face) */
    double vp[3];         /* particle velocity per axis at the step's start */
    double vf[3];         /* the larger face velocity magnitude per axis */
    double t;             /* time at the start of the step */
    int32_t particle, cell;
    int8_t face[3];       /* +1 high face, -1 low face, 0 none */
    int8_t ax;            /* axis of the exit taken; -1 none (stop time, capture, no exit) */
    uint8_t pad[4];
} orc_trace_rec;

typedef struct {
    int32_t* cell; double *px, *py, *pz; double *gx, *gy, *gz; double* t;
    uint8_t* status; uint32_t* steps; uint8_t* exit_face; uint64_t* hash;
    /* timeseries [n_times][n]; ts_x == NULL disables */
    double *ts_x, *ts_y, *ts_z; int32_t* ts_cell; uint8_t* ts_status;
    /* pathline points, appended in the order produced; path == NULL disables;
     * *path_n counts every point, also those beyond path_cap */
    orc_path_rec* path; int64_t path_cap; int64_t* path_n;
    /* per-step trace (diagnostics: where two evaluations of one path part);
     * trace == NULL disables; *trace_n counts every step */
    struct orc_trace_rec* trace; int64_t trace_cap; int64_t* trace_n;
} orc_track_out;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_log1p(double x);
double orc_expm1(double w);
double orc_div(double d, double v);
double orc_exit_time(double v1, double v2, double A, double iA, double D, double p, int* face);
double orc_move(double v1, double A, double iA, double D, double p, double dt);
double orc_exit_time_plain(double v1, double v2, double A, double D, double p, int* face);
double orc_move_plain(double v1, double A, double D, double p, double dt);
int orc_release_box(const orc_field* f, int64_t n, const double lo[3], const double hi[3],
                    uint64_t seed, uint64_t id_offset,
                    int32_t* cell, double* px, double* py, double* pz, uint8_t* status);
int orc_release_explicit(const orc_field* f, int64_t n, const int32_t* cell_in, const double* frac,
                         int32_t* cell, double* px, double* py, double* pz, uint8_t* status);
/* steps0/hash0/face0 (each may be NULL): cell-steps already taken, the FNV
 * hash of the cells visited so far and the last face crossed, carried by a
 * resumed particle; the run continues them (a particle with steps0 == 0
 * starts a new hash). */
int orc_track(const orc_field* f, int64_t n,
              const int32_t* cell0, const double* px0, const double* py0, const double* pz0,
              const double* t0, const uint8_t* status0, const uint32_t* steps0, const uint64_t* hash0,
              const uint8_t* face0, const orc_track_opts* opt, const orc_track_out* out);
int orc_usg_track(const orc_usg_field* u, int64_t n,
                  const int32_t* cell0, const double* px0, const double* py0, const double* pz0,
                  const double* t0, const uint8_t* status0, const uint32_t* steps0, const uint64_t* hash0,
                  const uint8_t* face0, const orc_track_opts* opt, const orc_track_out* out);
int orc_usg_release_explicit(const orc_usg_field* u, int64_t n, const int32_t* cell_in, const double* frac,
                             int32_t* cell, double* px, double* py, double* pz, uint8_t* status);
#endif
