/*
 * mp.h - C ABI of libmp: semi-analytical particle tracking (Pollock 1988)
 * through a steady, structured, MODFLOW-style flow field on one GPU.
 *
 * The operation is the particle loop of the paper (Methods, "MODPATH" and
 * Fig. 1): every particle is moved independently, one displacement per cell,
 * from its position to a face of the current cell and across it into the
 * neighbour, until a stopping condition holds (a boundary face, the maximum
 * tracking time, a sink cell; Methods, "MODPATH").  Endpoint and timeseries
 * outputs follow the paper's simulation types (Methods, "MODPATH").
 *
 * Conventions used by every call:
 *   - grid nlay x nrow x ncol, cell (k, i, j), linear index
 *     c = (k * nrow + i) * ncol + j;
 *   - x runs along column j, y along row i, z along layer k (z grows with k);
 *   - face flows are signed positive in the +axis direction:
 *     qx[k][i][j] (j = 0..ncol) is the flow through the west face of column j,
 *     qy[k][i][j] (i = 0..nrow), qz[k][i][j] (k = 0..nlay); units m^3/s;
 *   - ibound: 0 inactive, 1 active, -1 constant head, 2 strong sink;
 *   - global positions are metres from origin + cumulative cell sizes.
 *
 * Ownership: the library owns every device buffer it allocates (fields,
 * groups, request outputs) and frees it in the matching *_free call.  Callers
 * own every host buffer they pass; inputs are copied during the call unless
 * MP_DEVICE_PTR says they are device pointers, which are then read during the
 * call only (field load, release) and never retained.
 *
 * Errors: every call returns MP_OK (0) or a negative MP_ERR_* code and leaves
 * its out-parameters untouched on error; mp_last_error() returns a message for
 * the calling thread's last failure.  No call aborts the process and no
 * device wait is unbounded.
 *
 * Threads: calls on one context are serialised internally; handles may be
 * used from any thread.
 */
#ifndef MP_H
#define MP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define MP_OK 0
#define MP_ERR_INVALID_ARG -1  /* null pointer, bad enum, bad size            */
#define MP_ERR_SHAPE -2        /* grid dimensions / array sizes inconsistent  */
#define MP_ERR_NONFINITE -3    /* NaN/Inf flow, porosity <= 0 in active cell */
#define MP_ERR_OOM -4          /* device allocation failed                    */
#define MP_ERR_BUSY -5         /* request still running (try again)          */
#define MP_ERR_TIMEOUT -6      /* mp_wait timed out; the request continues    */
#define MP_ERR_CUDA -7         /* a CUDA runtime call failed                  */
#define MP_ERR_NOT_READY -8    /* unknown or freed request id                 */
#define MP_ERR_DEVICE -9       /* a kernel raised its error flag (bad index)  */

/* ---- particle status (endpoint and timeseries records) -------------------- */
#define MP_ST_ACTIVE 0          /* still moving (timeseries rows only)        */
#define MP_ST_TIME 1            /* reached t_stop inside a cell               */
#define MP_ST_SINK 2            /* entered (or released in) a strong sink     */
#define MP_ST_BOUNDARY 3        /* next cell inactive or constant head        */
#define MP_ST_EXIT_DOMAIN 4     /* left the grid through an outer face        */
#define MP_ST_NO_EXIT 5         /* no reachable face and t_stop infinite      */
#define MP_ST_STEP_CAP 6        /* max_steps cell-steps taken                 */
#define MP_ST_INVALID_RELEASE 7 /* released outside the grid / in CH/inactive */
#define MP_N_STATUS 8

#define MP_FACE_NONE 255 /* exit_face: 0 x-, 1 x+, 2 y-, 3 y+, 4 z-, 5 z+ */

/* ---- enums and flags ------------------------------------------------------ */
#define MP_DEVICE_PTR 1u        /* array arguments are device pointers       */

#define MP_PREC_FP64 0          /* IEEE double throughout                     */
#define MP_PREC_MIXED 1         /* FP32 in-cell coordinates and velocities,
                                   travel time as an FP32 pair (~48 bits),
                                   FP64 output times and global positions    */
#define MP_PREC_MIXED_F64T 2    /* as MP_PREC_MIXED, with FP64 kept for the
                                   cumulative travel time and for the
                                   near-zero branch of the exit time
                                   (log1p(z)/z in FP64): the accuracy
                                   reference of the FP32 pair and series;
                                   rectilinear grids, not in graphs or
                                   mp_track_noalloc                          */

#define MP_MODE_ENDPOINT 1      /* bit: endpoint record per particle          */
#define MP_MODE_TIMESERIES 2    /* bit: a record per output time per particle */
#define MP_MODE_PATHLINE 4      /* bit: a point at release and one per cell-step */

#define MP_SCHED_STATIC 0       /* one thread per particle, plain grid        */
#define MP_SCHED_DYNAMIC 1      /* persistent warps refilled from a queue     */
#define MP_SCHED_AUTO 2         /* the context's tuned launch (mp_autotune)
                                   for this field, precision and mode, else
                                   dynamic, 128 threads, 4 steps per fetch   */

#define MP_TRACK_UPDATE_GROUP 1u /* write final state back into the group     */
#define MP_TRACK_PASS_WEAK_SINKS 2u /* enter sink cells and leave them through
                                   a reachable face; a particle that has none
                                   inside a sink cell is captured (SINK)
                                   (the paper's second test case lets
                                   particles pass through weak sinks).  With
                                   mp_track_opts.weak_sink_fraction f > 0 a
                                   sink cell still stops particles (SINK, on
                                   the face, as a strong sink) when its sink
                                   extracts at least f of the cell's inflow:
                                   (inflow - outflow) / inflow over the face
                                   flows, summed face by face in the order
                                   x-, x+, y-, y+, z-, z+ (a quadtree face:
                                   its sub-faces summed in list order); a
                                   cell without inflow extracts all of it */

#define MP_RELEASE_EXPLICIT 0
#define MP_RELEASE_BOX 1

typedef struct mp_ctx mp_ctx;
typedef struct mp_field mp_field;
typedef struct mp_group mp_group;
typedef struct mp_graph mp_graph;
typedef int64_t mp_req;

/* Flow field.  delr/delc/dz are always host arrays; qx..ibound are host
 * arrays unless flags has MP_DEVICE_PTR.  Sizes: qx nlay*nrow*(ncol+1),
 * qy nlay*(nrow+1)*ncol, qz (nlay+1)*nrow*ncol, porosity and ibound
 * nlay*nrow*ncol (row-major as in the linear cell index). */
typedef struct {
    int32_t nlay, nrow, ncol;
    const double* delr;      /* [ncol] cell widths along x (m), > 0   */
    const double* delc;      /* [nrow] cell widths along y (m), > 0   */
    const double* dz;        /* [nlay] cell thickness along z (m), > 0 */
    double origin[3];        /* global coordinates of face (0,0,0)    */
    const double* qx;
    const double* qy;
    const double* qz;
    const double* porosity;  /* (0, 1] in active and sink cells       */
    const int8_t* ibound;
    uint32_t flags;          /* MP_DEVICE_PTR                          */
} mp_field_desc;

/* Particle release.  kind MP_RELEASE_EXPLICIT: cell[n] linear indices and
 * local[n][3] fractions in [0,1] of the cell size per axis (clamped), t0[n]
 * start times or NULL for 0.  kind MP_RELEASE_BOX: n positions uniform in the
 * box [lo, hi] (global m; lo == hi on an axis gives a plane), drawn with
 * Philox4x32-10 keyed by seed, particle q using counter (q + id_offset, 0|1);
 * start time 0.  A particle released outside the grid or in an inactive or
 * constant-head cell gets status MP_ST_INVALID_RELEASE, one released in a
 * sink cell MP_ST_SINK; both take no steps. */
typedef struct {
    int64_t n;
    int32_t kind;
    uint32_t flags;          /* MP_DEVICE_PTR for cell/local/t0 */
    const int32_t* cell;
    const double* local;
    const double* t0;
    double lo[3], hi[3];
    uint64_t seed, id_offset;
} mp_release_desc;

/* Tracking options.  times[n_times] ascending (host); t_stop may be +inf
 * (endpoint mode then runs until every particle terminates or hits
 * max_steps).  block / steps_per_fetch: 0 picks the tuned default. */
typedef struct {
    int32_t mode;            /* MP_MODE_* bits                  */
    int32_t precision;       /* MP_PREC_*                       */
    int32_t schedule;        /* MP_SCHED_*                      */
    int32_t n_times;
    const double* times;
    double t_stop;
    int64_t max_steps;       /* <= 0: 1,000,000; counted since release */
    int32_t block;           /* threads per block, 0 = auto     */
    int32_t steps_per_fetch; /* dynamic schedule, 0 = auto      */
    uint32_t flags;          /* MP_TRACK_* bits                 */
    int64_t path_capacity;   /* pathline points the request keeps; <= 0: 64 per particle */
    double weak_sink_fraction; /* in [0, 1]; > 0 with MP_TRACK_PASS_WEAK_SINKS: a sink
                                  cell whose sink extracts at least this fraction of
                                  its inflow still stops particles (see below) */
} mp_track_opts;

/* Endpoint arrays (SoA, particle order).  Any pointer may be NULL to skip
 * that array.  cell is the last cell the particle was tracked in; for
 * SINK/BOUNDARY/EXIT_DOMAIN it sits on the face exit_face of that cell.
 * px/py/pz are offsets (m) from the cell's low faces; x/y/z global (m).
 * hash is FNV-1a (64-bit, over the 32-bit cell indices) of the sequence of
 * cells tracked in, release cell first.  steps, hash and exit_face count
 * from the release: a group resumed with MP_TRACK_UPDATE_GROUP carries
 * them, so a resumed run reports what one continued run would (plus one
 * partial step per pause). */
typedef struct {
    int32_t* cell;
    double *x, *y, *z;
    double *px, *py, *pz;
    double* t;
    uint8_t* status;
    uint32_t* steps;
    uint8_t* exit_face;
    uint64_t* hash;
} mp_endpoints;

/* One timeseries record; the output is [n_times][n] records, 32 bytes each.
 * status MP_ST_ACTIVE while moving; after termination the record holds the
 * final position and the final status. */
typedef struct {
    double x, y, z;
    int32_t cell;
    uint8_t status;
    uint8_t pad[3];
} mp_ts_record;

/* One pathline point (Methods, "MODPATH": pathline simulations record the
 * path of every particle), 48 bytes: the release point (seq = steps taken
 * before this request, status as released) and the point every cell-step
 * ends at: the entry point of the next cell (status ACTIVE), or where the
 * path stops (TIME on the stop time, or the final status).  Points are
 * stored in the order the GPU produces them (the points of one particle in
 * increasing seq, particles interleaved), as the paper's threads append to
 * their output units. */
typedef struct {
    double x, y, z, t;       /* global position (m), time (s)              */
    int32_t particle;        /* index in the group                         */
    int32_t cell;            /* cell after the step                        */
    uint32_t seq;            /* cell-steps since release                   */
    uint8_t status;          /* MP_ST_*                                    */
    uint8_t pad[3];
} mp_path_record;

typedef struct {
    uint64_t cell_steps;             /* sum of per-particle cell-steps   */
    uint64_t n_status[MP_N_STATUS];  /* particles per final status       */
    float kernel_ms;                 /* device time of the tracking kernel */
    int32_t device_error;            /* kernel error flag (0 = none)     */
    uint64_t path_points;            /* pathline points produced (also beyond
                                        the capacity: rerun with more room)  */
    uint64_t t_begin_ns, t_end_ns;   /* the tracking launch's window on the
                                        device's global timer (ns): earliest
                                        block start, latest block end (a
                                        batch's requests share their launch's;
                                        over all launches of mp_track_periods);
                                        0 when nothing was launched          */
} mp_stats;

/* Context on one CUDA device.  The device is made current on the calling
 * thread.  Errors: MP_ERR_INVALID_ARG, MP_ERR_CUDA. */
/* Passage: none (infrastructure: a context binds the library to one GPU; the paper runs its
 * particle loop on one desktop computer, Methods, "Synthetic test cases"). */
int mp_ctx_create(int device, mp_ctx** out);
/* Frees every field, group, request and graph still owned by the context
 * (waiting, bounded, for their work).  Errors: MP_ERR_INVALID_ARG (NULL). */
/* Passage: none (infrastructure). */
int mp_ctx_destroy(mp_ctx* ctx);

/* Message for this thread's last failed call ("" if none); the string is
 * owned by the library and valid until the thread's next failing call.
 * Never fails. */
/* Passage: none (infrastructure; thread-local and context-free, so it also reports failures of
 * calls that had no context). */
const char* mp_last_error(void);

/* Copy (or read, MP_DEVICE_PTR) a flow field and build its device form:
 * per-cell velocity records in FP64 and FP32 (the paper's central flow-data
 * object, Methods, "Multiprocessing"), neighbour classes and face
 * coordinates.  Validates shapes, finiteness and porosity.  Synchronous.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_SHAPE, MP_ERR_NONFINITE, MP_ERR_OOM,
 * MP_ERR_CUDA. */
/* Passage: Methods, "MODPATH" (the tracking reads the flow model's cell data) and
 * "Multiprocessing" (flow-related arrays stored once, centrally, reached through a pointer). */
int mp_field_load(mp_ctx* ctx, const mp_field_desc* d, mp_field** out);
/* Passage: none (infrastructure). */
int mp_field_free(mp_field* f);

/* Volume balance of a loaded field (rectilinear or quadtree), computed once
 * when it is loaded from its face flows (the face totals the velocities use):
 * per cell, inflow = the flow entering through its faces and outflow = the
 * flow leaving, summed face by face in the order x-, x+, y-, y+, z-, z+.
 * Pollock's method assumes every active cell conserves volume; a sink cell
 * extracts inflow - outflow.  All sums in cell order. */
typedef struct {
    double max_abs_residual;  /* active cells (ibound 1): max |inflow - outflow| (m^3/s) */
    int64_t max_abs_cell;     /* the first active cell with that residual; -1: none */
    double max_rel_residual;  /* active cells with inflow: max |inflow - outflow| / inflow */
    double sink_extraction;   /* sink cells (ibound 2): sum of inflow - outflow (m^3/s) */
    int64_t active_cells;
    int64_t sink_cells;
} mp_balance;

/* Errors: MP_ERR_INVALID_ARG (NULL). */
/* Passage: none (a check of the input: the tracking assumes the converged, volume-conserving flow
 * solution of Methods, "Synthetic test cases"). */
int mp_field_balance(const mp_field* f, mp_balance* out);

/* A rectangular unstructured (quadtree) grid: the paper's TC2 also runs on
 * a quadtree refinement of its grid.  Cells are axis-aligned boxes; each
 * face (x-, x+, y-, y+, z-, z+) of cell c has the sub-faces
 * face_off[6c + f] .. face_off[6c + f + 1] - 1, each with the neighbour
 * across it (nbr, -1 outside the domain), the flow through it (q, m^3/s,
 * positive along +axis) and its rectangle in the two other axes (rect[4]:
 * lo_a, hi_a, lo_b, hi_b, global m; the other axes in x, y, z order).  Every
 * connection is listed from both cells.  Host arrays (MP_DEVICE_PTR is not
 * accepted).  Pollock's displacement uses each face's total flow over the
 * cell's own face area; a particle leaving through a face enters the
 * neighbour of the sub-face holding its exit point when that sub-face's
 * flow runs with the crossing, else of the nearest one whose flow does
 * (the point moves onto it).  Tracking: FP64 only, explicit releases
 * (mp_release_group with MP_RELEASE_EXPLICIT), every mode (endpoint,
 * timeseries, pathline), batches and flow periods (fields with the same
 * boxes and sub-face layout).  Errors: MP_ERR_INVALID_ARG, MP_ERR_SHAPE,
 * MP_ERR_NONFINITE, MP_ERR_OOM, MP_ERR_CUDA. */
typedef struct {
    int64_t ncell;
    const double* box;        /* [ncell][6]: x0, y0, z0, dx, dy, dz (m), sizes > 0 */
    const double* porosity;   /* [ncell], in (0, 1] for active cells */
    const int8_t* ibound;     /* [ncell]: 0 inactive, 1 active, -1 constant head, 2 sink */
    const int64_t* face_off;  /* [6 ncell + 1], non-decreasing, face_off[0] = 0 */
    const int32_t* nbr;       /* [nsub] */
    const double* q;          /* [nsub] */
    const double* rect;       /* [nsub][4] */
    uint32_t flags;           /* 0 */
} mp_usg_desc;

/* Passage: Methods, "MODPATH" (structured and rectangular unstructured grids) and Results, "Grid
 * complexity" (TC2 on a quadtree refinement). */
int mp_usg_field_load(mp_ctx* ctx, const mp_usg_desc* d, mp_field** out);
/* Device bytes held by a loaded field.  Errors: MP_ERR_INVALID_ARG (NULL). */
/* Passage: none (infrastructure). */
int mp_field_bytes(const mp_field* f, size_t* bytes);

/* Create a particle group on the field (state resident on the device).
 * Runs on `stream` (a cudaStream_t, NULL = legacy default) and returns when
 * the release is enqueued; the state is ready in stream order.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_OOM, MP_ERR_CUDA. */
/* Passage: Methods, "Synthetic test cases" (particles injected uniformly at x_o in TC1; TC2
 * injects groups in stages) and Introduction (several particle groups). */
int mp_release_group(mp_ctx* ctx, const mp_field* f, const mp_release_desc* r, void* stream,
                     mp_group** out);
/* Passage: none (infrastructure). */
int mp_group_free(mp_group* g);
/* Passage: none (infrastructure). */
int mp_group_size(const mp_group* g, int64_t* n);

/* Track a group (Methods, "MODPATH": the particle loop) asynchronously on
 * `stream`.  Allocates the request's outputs (stream-ordered) and enqueues
 * the tracking kernel; returns the request id at once.  The group is read,
 * not changed, unless o->flags has MP_TRACK_UPDATE_GROUP (resume: the
 * group's state becomes the final state, terminated particles keep their
 * status).  A moving particle whose cell is inactive or constant-head under
 * the group's field ends there (BOUNDARY, no step), in a sink cell (SINK)
 * unless MP_TRACK_PASS_WEAK_SINKS lets that sink pass.
 * Errors: MP_ERR_INVALID_ARG (also: weak_sink_fraction outside [0, 1]),
 * MP_ERR_OOM, MP_ERR_CUDA. */
/* Passage: Introduction and Methods, "MODPATH" (the particle loop: one displacement per cell,
 * hand-over to the neighbour, the stopping conditions; endpoint, timeseries and pathline
 * simulations). */
int mp_track(mp_ctx* ctx, mp_group* g, const mp_track_opts* o, void* stream, mp_req* out);

/* Rebind a group to another field on the same grid (same dims, cell sizes
 * and origin; flows, porosity and ibound may differ): the next flow period
 * of a piecewise-steady model.  Requests already enqueued keep the field
 * they were launched with.  Not concurrent with mp_track on the same group.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_SHAPE (another grid). */
/* Passage: Methods, "MODPATH" (the time step loop updates the flow arrays at ts_max). */
int mp_group_set_field(mp_group* g, const mp_field* f);

/* Piecewise-steady (transient) flow (Methods, "MODPATH": the outermost loop
 * runs over the flow model's time steps and updates the flow arrays when a
 * step's end time is reached; TC2 runs three stress periods).
 * fields[p] (n_periods of them, all on the group's grid) holds from
 * t_end[p-1] to t_end[p]; t_end has n_periods - 1 ascending finite entries
 * (NULL when n_periods == 1) and the last field has no end.  One request:
 * one kernel launch per period on `stream`, each resuming from the state
 * the previous one left (particles stopped at a period end continue in the
 * next field, in the same cell; see mp_track for cells that change class).
 * Outputs as mp_track's: endpoints of every particle (from the period it
 * ended in), timeseries over o->times across the periods, stats summed
 * (cell_steps of all launches, each particle counted once by its final
 * status; kernel_ms from the first launch to the last).  The group changes
 * only with MP_TRACK_UPDATE_GROUP, which also rebinds it to the last field.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_SHAPE, MP_ERR_NONFINITE, MP_ERR_OOM,
 * MP_ERR_CUDA. */
/* Passage: Methods, "MODPATH" (the time step loop over the flow model's stress periods). */
int mp_track_periods(mp_ctx* ctx, mp_group* g, int n_periods, const mp_field* const* fields, const double* t_end,
                     const mp_track_opts* o, void* stream, mp_req* out);

/* Track several groups (fewer than 2^24) in one launch per precision: the particles of all
 * groups form one index space handed out by the persistent work queue (or
 * one thread each), the GPU form of the paper's dynamic schedule over one
 * particle loop (Methods, "Multiprocessing"; Results, "Thread scheduling").
 * groups[n] must share one field; opts[n] are per request (mode, times,
 * t_stop, max_steps, flags); schedule, block and steps_per_fetch of a launch
 * come from the first request of that precision.  out[n] receives request
 * ids that behave as mp_track's (own outputs and counters; kernel_ms is the
 * shared launch's time).  Errors: as mp_track; on error no request exists. */
/* Passage: Methods, "Multiprocessing" (dynamic scheduling of one particle loop) and Results,
 * "Thread scheduling". */
int mp_track_batch(mp_ctx* ctx, int n, mp_group* const* groups, const mp_track_opts* opts, void* stream,
                   mp_req* out);

/* Launch configuration chosen by the autotuner. */
typedef struct {
    int32_t schedule;         /* MP_SCHED_STATIC or MP_SCHED_DYNAMIC */
    int32_t block;
    int32_t steps_per_fetch;
    int32_t tried;            /* configurations timed */
    float ms;                 /* best time of the timed sample */
} mp_tuning;

/* Time candidate launch configurations (static and dynamic schedule x block
 * 64/128/256 x steps per fetch 1/4/16 for dynamic) on the first
 * min(n, sample) particles of the group (sample <= 0: all of them) with
 * options o (the group is not changed), keep the fastest in the context for (field, o->precision,
 * timeseries or not) and return it; later requests with MP_SCHED_AUTO use
 * it.  Synchronous (bounded waits).  The paper's scheduling study (Results,
 * "Thread scheduling") is this choice made by measurement.
 * Errors: as mp_track, MP_ERR_TIMEOUT. */
/* Passage: Results, "Thread scheduling" (the schedule chosen by measurement). */
int mp_autotune(mp_ctx* ctx, mp_group* g, const mp_track_opts* o, int64_t sample, void* stream, mp_tuning* out);

/* Install a launch configuration (e.g. one cached from an earlier run) for
 * (field, precision, timeseries).  Errors: MP_ERR_INVALID_ARG (NULL, a
 * schedule other than static or dynamic, block outside [32, 256], or a
 * negative steps per fetch). */
/* Passage: Results, "Thread scheduling" (a measured launch choice kept across runs). */
int mp_set_tuning(mp_ctx* ctx, const mp_field* f, int32_t precision, int32_t timeseries, const mp_tuning* t);

/* Captured batches (the batching pattern's CUDA graphs; the paper's many
 * particle groups, Conclusions).  n_reqs box-release requests on one field
 * (rel[i], kind MP_RELEASE_BOX) with their options (opts[i]; no
 * MP_TRACK_UPDATE_GROUP) become one CUDA graph: clear the counters, release
 * every group in one launch, track them in one batched launch per
 * precision.  Group state and outputs are allocated here, once; every
 * mp_graph_launch re-releases and re-tracks into them (one graph launch on
 * the stream instead of a host-side launch sequence).  The launch
 * configuration is fixed at capture (MP_SCHED_AUTO takes the tuned one).
 * Results are the same as mp_release_group + mp_track_batch with the same
 * descriptors.  Errors: MP_ERR_INVALID_ARG, MP_ERR_OOM, MP_ERR_CUDA. */
/* Passage: Introduction and Conclusions (simultaneous displacement of several particle groups).
 * */
int mp_graph_create(mp_ctx* ctx, const mp_field* f, int n_reqs, const mp_release_desc* rel,
                    const mp_track_opts* opts, void* stream, mp_graph** out);
/* Replace request i's box, seed and id offset for later launches (the
 * particle count is fixed: MP_ERR_SHAPE otherwise).  Ordered after earlier
 * work on `stream`; returns once the descriptor is on the device.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_SHAPE, MP_ERR_CUDA. */
/* Passage: Introduction and Conclusions (several particle groups). */
int mp_graph_set_release(mp_graph* g, int i, const mp_release_desc* rel, void* stream);
/* Replay the graph on `stream` (asynchronous).  Outputs of the previous
 * launch are overwritten: read them first (stream order).
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_CUDA. */
/* Passage: Introduction and Conclusions (several particle groups). */
int mp_graph_launch(mp_graph* g, void* stream);
/* The request ids (n_reqs of them) through which a launch's outputs are
 * read with mp_wait, mp_get_endpoints, mp_get_timeseries, mp_get_pathlines
 * and mp_get_stats (kernel_ms then spans the whole graph).  They belong to
 * the graph: mp_req_free refuses them, mp_graph_free releases them.
 * ids has room for n_reqs entries.  Errors: MP_ERR_INVALID_ARG (NULL). */
/* Passage: none (infrastructure). */
int mp_graph_requests(const mp_graph* g, mp_req* ids);
/* Waits (bounded) for the last launch, then frees everything the graph
 * holds.  The field must outlive the graph.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_TIMEOUT (then nothing is freed). */
/* Passage: none (infrastructure). */
int mp_graph_free(mp_graph* g);

/* Wait up to timeout_us microseconds (< 0: no limit is not offered; the
 * wait is always bounded, and a negative value means 60 s) for a request.
 * Errors: MP_ERR_TIMEOUT (still running), MP_ERR_NOT_READY (unknown id),
 * MP_ERR_DEVICE (kernel error flag), MP_ERR_CUDA. */
/* Passage: none (infrastructure: the paper's loop runs synchronously; here a request is awaited
 * with a bound). */
int mp_wait(mp_ctx* ctx, mp_req r, int64_t timeout_us);

/* 1 if the request's work has finished, 0 if not; negative on error. */
/* Passage: none (infrastructure). */
int mp_query(mp_ctx* ctx, mp_req r);

/* Copy endpoint arrays out.  flags & MP_DEVICE_PTR: destinations are device
 * pointers, copies are enqueued on `stream` after the request and the call
 * returns at once; otherwise destinations are host memory and the call
 * waits (bounded, 60 s) for the request and the copies.
 * Errors: MP_ERR_NOT_READY, MP_ERR_TIMEOUT, MP_ERR_CUDA. */
/* Passage: Methods, "MODPATH" (endpoint simulations) and "Synthetic test cases" (endpoint output
 * written after the outermost loop). */
int mp_get_endpoints(mp_ctx* ctx, mp_req r, const mp_endpoints* out, uint32_t flags, void* stream);

/* Copy the [n_times][n] timeseries records out (same rules as endpoints).
 * Errors: MP_ERR_INVALID_ARG (request has no timeseries), as above. */
/* Passage: Methods, "MODPATH" (timeseries simulations: particle positions at user-defined times)
 * and "Multiprocessing" (records written from inside the particle loop to thread-exclusive units).
 * */
int mp_get_timeseries(mp_ctx* ctx, mp_req r, mp_ts_record* out, uint32_t flags, void* stream);

/* Copy a pathline request's points (MP_MODE_PATHLINE) to host memory, or
 * to device memory with MP_DEVICE_PTR (then enqueued on `stream`): at most
 * max_points of them, in the order they were produced; *n_points gets the
 * number copied.  Points beyond the request's path_capacity are counted
 * (mp_stats.path_points) but not kept.  Waits (bounded) for the request.
 * Errors: MP_ERR_INVALID_ARG (no pathlines), MP_ERR_NOT_READY (unknown id),
 * MP_ERR_TIMEOUT, MP_ERR_DEVICE, MP_ERR_CUDA. */
/* Passage: Methods, "MODPATH" (pathline simulations) and "Multiprocessing" (records written from
 * inside the particle loop). */
int mp_get_pathlines(mp_ctx* ctx, mp_req id, mp_path_record* out, int64_t max_points, int64_t* n_points,
                     uint32_t flags, void* stream);

/* Device views of the request's own output buffers (valid until
 * mp_req_free); any out-pointer may be NULL.  The pointers are the
 * library's: read them in stream order after the request.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NOT_READY (unknown id). */
/* Passage: none (infrastructure). */
int mp_endpoints_device(mp_ctx* ctx, mp_req r, mp_endpoints* out, mp_ts_record** ts);

/* Counters of a finished request (waits, bounded, like mp_get_endpoints).
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NOT_READY (unknown id),
 * MP_ERR_TIMEOUT, MP_ERR_CUDA. */
/* Passage: Methods, "Multiprocessing" (counters summed over the parallel loop by a reduction); the
 * cell-step count is this library's work measure. */
int mp_get_stats(mp_ctx* ctx, mp_req r, mp_stats* out);

/* Release a request's outputs (stream-ordered after its work); the id is
 * unknown afterwards.  Errors: MP_ERR_INVALID_ARG (NULL, or a request
 * owned by a graph), MP_ERR_NOT_READY (unknown id). */
/* Passage: none (infrastructure). */
int mp_req_free(mp_ctx* ctx, mp_req r);

/* Device bytes mp_track allocates for n particles under options o (the
 * serving layer's admission uses it).  Errors: MP_ERR_INVALID_ARG. */
/* Passage: none (infrastructure for admitting particle groups, Conclusions). */
int mp_query_bytes(const mp_track_opts* o, int64_t n, size_t* bytes);

/* Number of CUDA kernel launches mp_track issues for these options (one
 * tracking launch per request; mp_track_periods: one per period).
 * Errors: MP_ERR_INVALID_ARG (NULL). */
/* Passage: none (infrastructure). */
int mp_track_launches(const mp_track_opts* o, int32_t* launches);

/* ---- host to host, transfers overlapped with tracking ----------------------
 * Track n particles given in host memory and write their results to host
 * memory in one call.  Release as mp_release_group with MP_RELEASE_EXPLICIT:
 * cell[n] (int32), local[3 n] (fractions in [0, 1]^3 of the cell's extent,
 * particle-major), t0[n] (release times; NULL: 0).  Results as
 * mp_get_endpoints (ep: any pointer may be NULL) and, when o->mode has
 * MP_MODE_TIMESERIES and ts is not NULL, the [n_times][n] records into
 * ts (row stride n).  Particles move independently (Methods, "MODPATH"), so
 * the call splits them into n_chunks contiguous chunks (n_chunks <= 0:
 * chunks of about 128 K particles, 2 to 16 of them) and runs chunk c's
 * copy-in, release, tracking and copy-out in order on the second of two
 * internal streams when c is odd, the first otherwise: the result copies of
 * one chunk overlap the tracking of the next.  MP_SCHED_AUTO runs the chunks
 * with the static schedule (its blocks retire as their particles finish, so
 * the next chunk's blocks take their SMs).  The results are those of one
 * mp_release_group + mp_track + mp_get_endpoints / mp_get_timeseries over
 * all n particles (bit for bit: the kernels are the same, particle by
 * particle).  Page-locked host buffers make the copies asynchronous;
 * pageable ones work, without the overlap.  The host arrays are owned by
 * the caller; the call returns after the last copy has landed (bounded
 * wait, 60 s) and frees what it allocated.  stats (may be NULL): the sums of
 * the chunks' counters; kernel_ms = device time from the first chunk's
 * start to the last chunk's last copy.  The two streams belong to the
 * context and are kept for its later calls (the chunks' buffers are then
 * reused in stream order); calls on one context run one at a time.
 * MP_MODE_PATHLINE is rejected.
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NONFINITE, MP_ERR_OOM, MP_ERR_TIMEOUT,
 * MP_ERR_DEVICE, MP_ERR_CUDA. */
/* Passage: Introduction and Methods, "MODPATH" (independent particles, so they can be tracked in
 * chunks). */
int mp_track_host(mp_ctx* ctx, const mp_field* f, int64_t n, const int32_t* cell, const double* local,
                  const double* t0, const mp_track_opts* o, int32_t n_chunks, const mp_endpoints* ep,
                  mp_ts_record* ts, mp_stats* stats);

/* ---- tracking without device allocation ----------------------------------
 * The paper has no counterpart of this call.  It exists for callers that
 * cannot allocate device memory where they track: code that runs inside a
 * memory budget it does not control (an embedding application that hands
 * out one fixed arena and forbids further cudaMalloc), or code that must not
 * let a library grow the device's memory pool behind its back.  The caller
 * passes every buffer: the particle state (device arrays in the layout of a
 * group: cell int32, px/py/pz offsets in m from the cell's low faces and t
 * as FP64, status u8), the endpoint arrays (device, all required) and, in
 * timeseries mode, the [n_times][n] record buffer (device).  times stays a
 * host array.  The call allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine.  Its only other device memory is a fixed
 * file-scope array of 8 + 13 + 2 * MP_NOALLOC_MAX_TIMES 64-bit words plus
 * the launch's request descriptor (queue head, counters, the output times in
 * FP64 and as FP32 pairs; about 66 KB) that every GPU that loads the library
 * holds until the process exits.
 *   - The call runs on the device of f's context and restores the caller's
 *     current device before it returns.
 *   - The first call on each device takes the array's device address
 *     (cudaGetSymbolAddress) and keeps it.
 *   - The output times and the request descriptor reach the device through
 *     cudaMemcpyAsync from pageable host memory, which may block the calling
 *     thread until `stream` reaches the copy.  A stream that is capturing is
 *     refused (MP_ERR_INVALID_ARG).
 *   - Every call shares the array, which keeps the last call's contents; the
 *     call clears the queue head and counters itself.  Calls that overlap on
 *     the GPU (different streams, or a second call before the first has run)
 *     race on it: run them one after another on one stream.
 *   - n_times > MP_NOALLOC_MAX_TIMES is rejected with MP_ERR_INVALID_ARG.
 *   - stats == NULL: the call returns once the work is enqueued on `stream`.
 *     Otherwise it waits for the stream and fills *stats (kernel_ms is 0).
 * Errors: MP_ERR_INVALID_ARG, MP_ERR_NONFINITE, MP_ERR_CUDA, MP_ERR_DEVICE. */
#define MP_NOALLOC_MAX_TIMES 4096

typedef struct {
    int64_t n;
    int32_t* cell;
    double *px, *py, *pz, *t;
    uint8_t* status;
    mp_endpoints out;
    mp_ts_record* ts;
    mp_track_opts opts;
} mp_noalloc_args;

/* Passage: none: the paper has no counterpart (see the block above). */
int mp_track_noalloc(const mp_field* f, const mp_noalloc_args* a, void* stream, mp_stats* stats);

#ifdef __cplusplus
}
#endif
#endif /* MP_H */
