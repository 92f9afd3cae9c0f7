// mp_internal.h - device-side layouts and kernel launchers of libmp.
//
// Field layout in HBM (built once by mp_field_load):
//   rec64[c]  128 B {v1x, Ax, iAx, v1y, Ay, iAy, v1z, Az, iAz, nb, FP32 copies}:
//             the FP64 low-face velocities v1 = Q1 / (n * area), gradients
//             A = (v2 - v1) / D of Pollock (1988) and iA = 1 / A (0 when
//             A == 0), one line per cell-step; the FP64 path needs only the
//             signs of v1 and v2 beyond these, kept as bits of nb.
//   rec32[c]  32 B  {u1x, u2x, u1y, u2y, u1z, u2z, nb, pad}: the same
//             velocities divided by the cell size (units 1/s) in FP32 for
//             the mixed-precision path, which works in local fractions
//             xi in [0, 1]; one 32-byte sector per cell-step.
//   nb        2 bits per face (x-, x+, y-, y+, z-, z+): the class of the
//             neighbour across it (0 active, 1 sink, 2 inactive or constant
//             head, 3 outside the grid), so crossing needs no second gather;
//             bits 16 + 4a .. 19 + 4a (axis a): v1 > 0, v1 < 0, v2 > 0, v2 < 0.
//   delr/delc/dz and face coordinates xf/yf/zf (n+1 entries each, FP64).
// Particle state (group) in SoA: cell int32, px/py/pz/t FP64, status u8.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp.h"

namespace mp {

enum : int { NB_ACTIVE = 0, NB_SINK = 1, NB_BOUNDARY = 2, NB_OUTSIDE = 3 };

enum : int { NB_SIGN = 16 };   // first face-velocity sign bit of nb

struct __align__(16) CellF64 {
    double v1x, Ax, iAx, v1y, Ay, iAy, v1z, Az, iAz;
    unsigned long long nb;
    // FP32 copies of the same values, for screening the exit axis
    float fv1x, fv2x, fAx, fv1y, fv2y, fAy, fv1z, fv2z, fAz;
    float pad[3];
};
static_assert(sizeof(CellF64) == 128, "CellF64 is one 128-byte line");

struct __align__(32) CellF32 {
    float u1x, u2x, u1y, u2y, u1z, u2z;
    uint32_t nb;
    float pad;
};
static_assert(sizeof(CellF32) == 32, "CellF32 is one 32-byte sector");

struct DevField {
    int nlay, nrow, ncol;
    long long ncell;
    const CellF64* rec64;
    const CellF32* rec32;
    const double* delr;
    const double* delc;
    const double* dz;
    const double* xf;  // [ncol+1]
    const double* yf;  // [nrow+1]
    const double* zf;  // [nlay+1]
    const int8_t* ibound;
    const double* sinkfrac;   // per cell: fraction of the inflow a sink cell extracts
    // x / ncol and x / nrow as a 64-bit multiply-high (x < 2^32):
    // floor(x / d) == umul64hi(x, floor((2^64 - 1) / d) + 1) for 1 < d < 2^32
    unsigned long long m_ncol, m_nrow;
};

__host__ __device__ inline unsigned long long div_magic(unsigned d)
{
    return d <= 1 ? 0ULL : (~0ULL) / d + 1ULL;
}

#ifdef __CUDACC__
__device__ __forceinline__ unsigned fast_div(unsigned x, unsigned d, unsigned long long m)
{
    return d <= 1 ? x : (unsigned)__umul64hi((unsigned long long)x, m);
}

// (k, i, j) of a linear cell index without integer division instructions
__device__ __forceinline__ void split_cell(const DevField& f, int c, int& k, int& i, int& j)
{
    const unsigned r = fast_div((unsigned)c, (unsigned)f.ncol, f.m_ncol);   // k * nrow + i
    j = c - (int)(r * (unsigned)f.ncol);
    k = (int)fast_div(r, (unsigned)f.nrow, f.m_nrow);
    i = (int)r - k * f.nrow;
}
#endif

struct DevState {
    int32_t* cell;
    double* px;
    double* py;
    double* pz;
    double* t;
    uint8_t* status;
    // carried by a resumed particle (each may be NULL: a fresh start)
    uint32_t* steps;             // cell-steps since release
    unsigned long long* hash;    // FNV hash of the cells visited (read when steps > 0)
    uint8_t* exit_face;          // last face crossed (read when steps > 0)
};

// status a later flow period gives a particle that had already ended: the
// launch neither writes nor counts it
enum : int { ST_SKIP = 0xFF };

// counters[0] = cell-steps, [1 + s] = particles with final status s,
// [COUNTER_ERR] = device error flag (index of the first bad access + 1),
// [COUNTER_T_BEGIN] / [COUNTER_T_END] = the launch's device-time window:
// the complement of the global timer (ns) at the earliest block start and
// the timer at the latest block end (both kept with atomicMax from zero)
enum : int {
    COUNTER_STEPS = 0,
    COUNTER_STATUS = 1,
    COUNTER_ERR = 1 + MP_N_STATUS,
    COUNTER_PATH = 2 + MP_N_STATUS,   // pathline points appended (the append cursor)
    COUNTER_T_BEGIN = 3 + MP_N_STATUS,
    COUNTER_T_END = 4 + MP_N_STATUS,
    N_COUNTERS = 5 + MP_N_STATUS
};

// launch modes: which outputs the kernel variant writes besides endpoints
enum : unsigned { MODE_TS = 1u, MODE_PATH = 2u };

struct DevOut {
    int32_t* cell;
    double* x;
    double* y;
    double* z;
    double* px;
    double* py;
    double* pz;
    double* t;
    uint8_t* status;
    uint32_t* steps;
    uint8_t* exit_face;
    unsigned long long* hash;
    mp_ts_record* ts;            // [n_times][n] or nullptr
    const double* times;         // device copy, [n_times]
    const float2* times_ff;      // the same times as FP32 pairs (hi, lo)
    unsigned long long* counters;  // [N_COUNTERS]
    mp_path_record* path;        // pathline points or nullptr
    long long path_cap;          // points that fit in path
};

struct TrackParams {
    long long n;
    double t_stop;
    long long max_steps;
    int n_times;
    int steps_per_fetch;
    int update_group;
    int pass_sinks;              // enter sink cells, leave through outflow faces
    double sink_frac;            // > 0 with pass_sinks: sinks extracting at least this fraction still stop
    int cont;                    // a later flow period of one request: skip ended particles and
                                 // output times already written
    int last;                    // the request's last launch: count particles paused at its stop time
    int pathline;                // append pathline points
    float tstop_hi, tstop_lo;    // t_stop as an FP32 pair (inf, 0 when infinite)
};

#ifdef __CUDACC__
// a sink cell with extraction fraction sf stops particles (entering it or
// resumed in it): always without pass-through, with it when sf >= sink_frac > 0
__device__ __forceinline__ bool sink_stops(const TrackParams& p, const double* sinkfrac, long long c)
{
    return !p.pass_sinks || (p.sink_frac > 0.0 && __ldg(sinkfrac + c) >= p.sink_frac);
}
#endif

// One tracking request of a launch: its particle state, outputs and options.
struct Req {
    DevState in;
    DevOut o;
    TrackParams p;
};

// A launch tracks the particles of one or more requests as one index space:
// global particle g belongs to request r with starts[r] <= g < starts[r+1].
struct Batch {
    const Req* reqs;             // [n_reqs], device
    const long long* starts;     // [n_reqs + 1], device
    int n_reqs;
    long long n_total;
    int steps_per_fetch;
    unsigned long long* queue;   // dynamic schedule head (zeroed before launch)
};

// split an FP64 value into an FP32 pair hi + lo (hi = round(v), lo = round(v - hi))
inline void split_ff(double v, float& hi, float& lo)
{
    hi = (float)v;
    lo = (v - (double)hi < 3.0e38 && v - (double)hi > -3.0e38) ? (float)(v - (double)hi) : 0.0f;
}

// Kernel launchers (each enqueues one kernel on `s`).
cudaError_t launch_validate(const double* qx, long long nqx, const double* qy, long long nqy, const double* qz,
                            long long nqz, const double* por, const int8_t* ib, long long ncell, unsigned* flags,
                            cudaStream_t s);
// Rectangular unstructured grid (device form, built by mp_usg_field_load):
//   cell[c]  128 B, the layout of CellF64: {v1x, Ax, iAx, v1y, Ay, iAy, v1z,
//            Az, iAz, sg, FP32 copies of v1, v2, A}: Pollock velocities from
//            each face's total flow (sub-faces summed in list order); sg
//            holds the face-velocity sign bits (bits 4a .. 4a + 3: v1 > 0,
//            v1 < 0, v2 > 0, v2 < 0)
//   geo[c]   48 B {low corner, sizes} of the box
//   face_off[6 c + f] .. face_off[6 c + f + 1] - 1: sub-faces of face f
//   sub[e]   48 B {neighbour (-1 outside), flow along +axis, rectangle in
//            the two other axes (lo_a, hi_a, lo_b, hi_b)}
using UsgCell = CellF64;

struct __align__(16) UsgGeo {
    double o[3];
    double D[3];
};

struct __align__(16) UsgSub {
    int nbr;
    int pad;
    double q;
    double rect[4];
};

struct DevUsg {
    long long ncell;
    long long nsub;
    const UsgCell* cell;
    const UsgGeo* geo;
    const long long* face_off;
    const UsgSub* sub;
    const int8_t* ibound;
    const double* sinkfrac;   // per cell: fraction of the inflow a sink cell extracts
};

cudaError_t launch_build_usg(const DevUsg& u, UsgCell* cell, UsgGeo* geo, double* sinkfrac, double2* inout,
                             const double* box, const double* por, cudaStream_t s);
cudaError_t launch_release_explicit_usg(const DevUsg& u, const DevState& st, long long n, const int32_t* cell,
                                        const double* local, const double* t0, cudaStream_t s);
cudaError_t launch_track_usg(const DevUsg& u, const Batch& b, unsigned modes, int schedule, int block,
                             int blocks_per_sm_cap, cudaStream_t s);

// one group's box release, as a device descriptor (graph replays read it)
struct BoxRelease {
    DevState st;
    long long n;
    double lo[3], hi[3];
    unsigned long long seed, id_offset;
};

cudaError_t launch_release_boxes(const DevField& f, const BoxRelease* d, const long long* starts, int n_reqs,
                                 long long n_total, cudaStream_t s);
cudaError_t launch_build_records(const DevField& f, CellF64* rec64, CellF32* rec32, double* sinkfrac,
                                 double2* inout, const double* qx, const double* qy, const double* qz,
                                 const double* por, cudaStream_t s);
cudaError_t launch_release_box(const DevField& f, const DevState& st, long long n, const double lo[3],
                               const double hi[3], unsigned long long seed, unsigned long long id_offset,
                               cudaStream_t s);
cudaError_t launch_release_explicit(const DevField& f, const DevState& st, long long n, const int32_t* cell,
                                    const double* local, const double* t0, cudaStream_t s);
// ts: true if any request of the batch writes timeseries records
cudaError_t launch_track_fp64(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                              int blocks_per_sm_cap, cudaStream_t s);
cudaError_t launch_track_mixed(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                               int blocks_per_sm_cap, cudaStream_t s);
// copy the first request's launch window into the other requests of a batch
cudaError_t launch_spread_window(const Batch& b, cudaStream_t s);
cudaError_t launch_track_mixed_f64t(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                               int blocks_per_sm_cap, cudaStream_t s);

// Host helpers shared by the entry points: the calling thread's error
// message (what mp_last_error returns) and a loaded field's device view.
void set_last_error(const char* msg);
const DevField* field_device_view(const mp_field* f);
bool field_is_usg(const mp_field* f);
int field_device(const mp_field* f);   // the device of the field's context

}  // namespace mp
