// mp_fp64.cu - field records, particle release and FP64 tracking kernels.
//
// Compiled with -fmad=false: every multiply and add below rounds on its own,
// in the order written, so that the FP64 path evaluates the same IEEE
// operations as a plain double-precision statement of the method.
//
// Method (Pollock 1988, the displacement scheme the paper keeps unchanged;
// Methods, "MODPATH"): inside a cell each velocity component varies linearly
// between its two faces, v(p) = v1 + A p with A = (v2 - v1) / D, so the
// motion along each axis is p(t) = p + v_p (e^{A t} - 1) / A (p + v_p t when
// A t == 0) and the time to reach the exit face is t_a = ln(1 + z) / A with
// z = A (d / v_p) (t_a = d / v_p when z == 0); 1 / A comes with the cell.  The particle leaves through the
// face with the smallest t_a (lowest axis on ties) and is handed to the
// neighbour across it, until a stopping condition holds (Methods, "MODPATH").
#include <cfloat>
#include <cmath>

#include "mp_internal.h"
#include "mp_sched.cuh"
#include "mp_f64math.cuh"

namespace mp {

// ---------------------------------------------------------------------------
// field records
// ---------------------------------------------------------------------------

__device__ __forceinline__ int nb_class(const DevField& f, int k, int i, int j)
{
    if (k < 0 || k >= f.nlay || i < 0 || i >= f.nrow || j < 0 || j >= f.ncol) return NB_OUTSIDE;
    const int8_t ib = f.ibound[((long long)k * f.nrow + i) * f.ncol + j];
    if (ib == 1) return NB_ACTIVE;
    if (ib == 2) return NB_SINK;
    return NB_BOUNDARY;
}

// a cell's inflow and outflow from its six face flows (+axis direction),
// face by face in the order x-, x+, y-, y+, z-, z+
__device__ double2 face_inout(const double q[6])
{
    double in = 0.0, out = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double q1 = q[2 * a], q2 = q[2 * a + 1];
        if (q1 > 0.0) in += q1; else out += -q1;
        if (q2 < 0.0) in += -q2; else out += q2;
    }
    return make_double2(in, out);
}

// fraction of a cell's inflow its sink extracts; no inflow: 1
__device__ double sink_fraction(double2 io)
{
    return io.x > 0.0 ? (io.x - io.y) / io.x : 1.0;
}

__global__ void k_build_records(DevField f, CellF64* r64, CellF32* r32, double* sinkfrac, double2* inout,
                                const double* qx, const double* qy, const double* qz, const double* por)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= f.ncell) return;
    const int ncol = f.ncol, nrow = f.nrow;
    const int j = (int)(c % ncol), i = (int)((c / ncol) % nrow), k = (int)(c / ((long long)ncol * nrow));
    unsigned long long nb = 0;
    nb |= (unsigned long long)nb_class(f, k, i, j - 1) << 0;
    nb |= (unsigned long long)nb_class(f, k, i, j + 1) << 2;
    nb |= (unsigned long long)nb_class(f, k, i - 1, j) << 4;
    nb |= (unsigned long long)nb_class(f, k, i + 1, j) << 6;
    nb |= (unsigned long long)nb_class(f, k - 1, i, j) << 8;
    nb |= (unsigned long long)nb_class(f, k + 1, i, j) << 10;
    CellF64 r{};
    CellF32 s{};
    double v2x = 0.0, v2y = 0.0, v2z = 0.0;
    const int8_t ib = f.ibound[c];
    if (ib == 1 || ib == 2) {
        const double n = por[c];
        const double dx = f.delr[j], dy = f.delc[i], dzz = f.dz[k];
        const double ax = dy * dzz, ay = dx * dzz, az = dx * dy;
        const double qx1 = qx[((long long)k * nrow + i) * (ncol + 1) + j];
        const double qx2 = qx[((long long)k * nrow + i) * (ncol + 1) + j + 1];
        const double qy1 = qy[((long long)k * (nrow + 1) + i) * ncol + j];
        const double qy2 = qy[((long long)k * (nrow + 1) + i + 1) * ncol + j];
        const double qz1 = qz[((long long)k * nrow + i) * ncol + j];
        const double qz2 = qz[((long long)(k + 1) * nrow + i) * ncol + j];
        r.v1x = qx1 / (n * ax); v2x = qx2 / (n * ax);
        r.v1y = qy1 / (n * ay); v2y = qy2 / (n * ay);
        r.v1z = qz1 / (n * az); v2z = qz2 / (n * az);
        r.Ax = (v2x - r.v1x) / dx;
        r.Ay = (v2y - r.v1y) / dy;
        r.Az = (v2z - r.v1z) / dzz;
        r.iAx = r.Ax != 0.0 ? 1.0 / r.Ax : 0.0;
        r.iAy = r.Ay != 0.0 ? 1.0 / r.Ay : 0.0;
        r.iAz = r.Az != 0.0 ? 1.0 / r.Az : 0.0;
        s.u1x = (float)(r.v1x / dx); s.u2x = (float)(v2x / dx);
        s.u1y = (float)(r.v1y / dy); s.u2y = (float)(v2y / dy);
        s.u1z = (float)(r.v1z / dzz); s.u2z = (float)(v2z / dzz);
        const double q6[6] = {qx1, qx2, qy1, qy2, qz1, qz2};
        const double2 io = face_inout(q6);
        inout[c] = io;
        if (ib == 2) sinkfrac[c] = sink_fraction(io);
    } else {
        inout[c] = make_double2(0.0, 0.0);
    }
    if (ib != 2) sinkfrac[c] = 0.0;
    const double v1a[3] = {r.v1x, r.v1y, r.v1z}, v2a[3] = {v2x, v2y, v2z};
    for (int a = 0; a < 3; ++a) {
        const unsigned long long sg = (v1a[a] > 0.0 ? 1ULL : 0ULL) | (v1a[a] < 0.0 ? 2ULL : 0ULL) |
                                      (v2a[a] > 0.0 ? 4ULL : 0ULL) | (v2a[a] < 0.0 ? 8ULL : 0ULL);
        nb |= sg << (NB_SIGN + 4 * a);
    }
    r.nb = nb;
    r.fv1x = (float)r.v1x; r.fv2x = (float)v2x; r.fAx = (float)r.Ax;
    r.fv1y = (float)r.v1y; r.fv2y = (float)v2y; r.fAy = (float)r.Ay;
    r.fv1z = (float)r.v1z; r.fv2z = (float)v2z; r.fAz = (float)r.Az;
    s.nb = (uint32_t)nb;
    r64[c] = r;
    r32[c] = s;
}

cudaError_t launch_build_records(const DevField& f, CellF64* rec64, CellF32* rec32, double* sinkfrac,
                                 double2* inout, const double* qx, const double* qy, const double* qz,
                                 const double* por, cudaStream_t s)
{
    if (f.ncell <= 0) return cudaSuccess;
    const int b = 256;
    const long long g = (f.ncell + b - 1) / b;
    k_build_records<<<(unsigned)g, b, 0, s>>>(f, rec64, rec32, sinkfrac, inout, qx, qy, qz, por);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// release: Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    #pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ double unit53(unsigned a, unsigned b)
{
    const unsigned long long v = ((((unsigned long long)a) << 32) | (unsigned long long)b) >> 11;
    return (double)v * (1.0 / 9007199254740992.0);
}

// largest a in [0, n-1] with f[a] <= x; -1 if x is outside [f[0], f[n]]
__device__ __forceinline__ int locate(const double* fc, int n, double x)
{
    if (!(x >= fc[0]) || !(x <= fc[n])) return -1;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fc[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint8_t release_status(const DevField& f, long long c)
{
    const int8_t ib = f.ibound[c];
    return ib == 1 ? MP_ST_ACTIVE : (ib == 2 ? MP_ST_SINK : MP_ST_INVALID_RELEASE);
}

struct Box { double lo[3], hi[3]; };

// one particle of a box release: Philox counters (id, 0) and (id, 1) under
// the key `seed`, three 53-bit uniforms, the cell holding the point
__device__ __forceinline__ void release_one(const DevField& f, const DevState& st, long long q, const Box& b,
                                            unsigned long long seed, unsigned long long off)
{
    const unsigned long long id = (unsigned long long)q + off;
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    const uint4 r = philox4x32_10(make_uint4((unsigned)id, (unsigned)(id >> 32), 0u, 0u), key);
    const uint4 s = philox4x32_10(make_uint4((unsigned)id, (unsigned)(id >> 32), 1u, 0u), key);
    const double ux = unit53(r.x, r.y), uy = unit53(r.z, r.w), uz = unit53(s.x, s.y);
    const double gx = b.lo[0] + ux * (b.hi[0] - b.lo[0]);
    const double gy = b.lo[1] + uy * (b.hi[1] - b.lo[1]);
    const double gz = b.lo[2] + uz * (b.hi[2] - b.lo[2]);
    const int j = locate(f.xf, f.ncol, gx), i = locate(f.yf, f.nrow, gy), k = locate(f.zf, f.nlay, gz);
    st.t[q] = 0.0;
    if (st.steps) st.steps[q] = 0u;
    if (j < 0 || i < 0 || k < 0) {
        st.cell[q] = -1; st.px[q] = 0.0; st.py[q] = 0.0; st.pz[q] = 0.0;
        st.status[q] = MP_ST_INVALID_RELEASE;
        return;
    }
    double ox = gx - f.xf[j], oy = gy - f.yf[i], oz = gz - f.zf[k];
    ox = fmin(fmax(ox, 0.0), f.delr[j]);
    oy = fmin(fmax(oy, 0.0), f.delc[i]);
    oz = fmin(fmax(oz, 0.0), f.dz[k]);
    const long long c = ((long long)k * f.nrow + i) * f.ncol + j;
    st.cell[q] = (int32_t)c;
    st.px[q] = ox; st.py[q] = oy; st.pz[q] = oz;
    st.status[q] = release_status(f, c);
}

__global__ void k_release_box(DevField f, DevState st, long long n, Box b, unsigned long long seed,
                              unsigned long long off)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    release_one(f, st, q, b, seed, off);
}

// Box releases of several groups in one launch: one index space over all
// of them (starts = prefix sums of the group sizes), the descriptors read
// from device memory, so a captured graph releases whatever they hold.
__global__ void k_release_boxes(DevField f, const BoxRelease* d, const long long* starts, int n_reqs,
                                long long n_total)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_total) return;
    int lo = 0, hi = n_reqs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    const BoxRelease& r = d[lo];
    Box b;
    for (int a = 0; a < 3; ++a) { b.lo[a] = r.lo[a]; b.hi[a] = r.hi[a]; }
    release_one(f, r.st, g - starts[lo], b, r.seed, r.id_offset);
}

cudaError_t launch_release_boxes(const DevField& f, const BoxRelease* d, const long long* starts, int n_reqs,
                                 long long n_total, cudaStream_t s)
{
    if (n_total <= 0) return cudaSuccess;
    k_release_boxes<<<(unsigned)((n_total + 255) / 256), 256, 0, s>>>(f, d, starts, n_reqs, n_total);
    return cudaGetLastError();
}

__global__ void k_release_explicit(DevField f, DevState st, long long n, const int32_t* cell,
                                   const double* local, const double* t0)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long c = cell[q];
    st.t[q] = t0 ? t0[q] : 0.0;
    if (c < 0 || c >= f.ncell) {
        st.cell[q] = -1; st.px[q] = 0.0; st.py[q] = 0.0; st.pz[q] = 0.0;
        st.status[q] = MP_ST_INVALID_RELEASE;
        return;
    }
    const int j = (int)(c % f.ncol), i = (int)((c / f.ncol) % f.nrow), k = (int)(c / ((long long)f.ncol * f.nrow));
    const double fx = fmin(fmax(local[3 * q], 0.0), 1.0);
    const double fy = fmin(fmax(local[3 * q + 1], 0.0), 1.0);
    const double fz = fmin(fmax(local[3 * q + 2], 0.0), 1.0);
    st.cell[q] = (int32_t)c;
    st.px[q] = fx * f.delr[j]; st.py[q] = fy * f.delc[i]; st.pz[q] = fz * f.dz[k];
    st.status[q] = release_status(f, c);
}

cudaError_t launch_release_box(const DevField& f, const DevState& st, long long n, const double lo[3],
                               const double hi[3], unsigned long long seed, unsigned long long id_offset,
                               cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    Box b;
    for (int a = 0; a < 3; ++a) { b.lo[a] = lo[a]; b.hi[a] = hi[a]; }
    k_release_box<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, st, n, b, seed, id_offset);
    return cudaGetLastError();
}

cudaError_t launch_release_explicit(const DevField& f, const DevState& st, long long n, const int32_t* cell,
                                    const double* local, const double* t0, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_release_explicit<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, st, n, cell, local, t0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 tracking engine
// ---------------------------------------------------------------------------

struct F64Engine {
    // blocks of 256 threads to keep resident per SM (0: no target; the
    // kernels are FP64-pipe bound)
    static constexpr int min_blocks(bool, bool, bool) { return 0; }
    DevField f;
    Batch b;

    struct State {
        int r;            // request of the particle within the launch
        int c, i, j, k;
        double x0, x1, x2;   // offsets (m) from the cell's low faces
        double t;
        unsigned steps;
        unsigned long long h;
        int kn;
        int st;
        int ef;
        int in_sink;      // the current cell is a sink entered with pass-through
        double tev;  // next output time or the stop time, whichever is first
    };

    __device__ __forceinline__ static int face_of(double vp, bool v2pos, bool v1neg)
    {
        return f64_face(vp, v2pos, v1neg);
    }

    // face-velocity signs of axis a from the cell's nb word
    __device__ __forceinline__ static bool v1_neg(unsigned long long nb, int a)
    {
        return (nb >> (NB_SIGN + 4 * a + 1)) & 1ULL;
    }
    __device__ __forceinline__ static bool v2_pos(unsigned long long nb, int a)
    {
        return (nb >> (NB_SIGN + 4 * a + 2)) & 1ULL;
    }

    template <class T>
    __device__ __forceinline__ static T sel3(int a, T x, T y, T z)
    {
        return a == 0 ? x : (a == 1 ? y : z);
    }

    __device__ __forceinline__ static float estimate(int face, float d, double vp, float fA, float fue, bool& unsafe)
    {
        return f32_estimate_f(face, d, vp, fA, fue, unsafe);
    }

    __device__ __forceinline__ static double move(double A, double iA, double D, double vp, double pp, double dt)
    {
        return f64_move(A, iA, D, vp, pp, dt);
    }

    __device__ __forceinline__ void record(long long q, int kk, const State& s, double x, double y, double z,
                                           int st) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        store_record(o.ts + (long long)kk * p.n + q, x, y, z, s.c, st);
    }

    __device__ __forceinline__ double gx(const State& s) const { return __ldg(f.xf + s.j) + s.x0; }
    __device__ __forceinline__ double gy(const State& s) const { return __ldg(f.yf + s.i) + s.x1; }
    __device__ __forceinline__ double gz(const State& s) const { return __ldg(f.zf + s.k) + s.x2; }

    __device__ __forceinline__ void final_pos(const State& s, double& x, double& y, double& z) const
    {
        const bool ok = s.c >= 0;
        x = ok ? gx(s) : CUDART_NAN;
        y = ok ? gy(s) : CUDART_NAN;
        z = ok ? gz(s) : CUDART_NAN;
    }

    // next time at which the step loop must leave its fast path
    __device__ __forceinline__ double next_event(const State& s) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        const double tk = s.kn < p.n_times ? __ldg(o.times + s.kn) : CUDART_INF;
        // fmin on the integer side: only the lanes with output times in the
        // step take this, and an FP64 compare would hold the whole warp's
        // FP64 pipe slot for them
        return ge_d(tk, p.t_stop) ? p.t_stop : tk;
    }

    template <bool TS>
    __device__ __forceinline__ void load(int r, long long q, State& s) const
    {
        s.r = r;
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        s.c = in.cell[q];
        s.st = in.status[q];
        // a later flow period leaves particles that ended before it untouched
        // (decided on the stored status, before this field's cell classes)
        if (p.cont && s.st != MP_ST_ACTIVE) {
            s.st = ST_SKIP;
            return;
        }
        s.x0 = in.px[q]; s.x1 = in.py[q]; s.x2 = in.pz[q];
        s.t = in.t[q];
        // cell-steps, hash and last face carried by a resumed particle
        s.steps = in.steps ? in.steps[q] : 0u;
        s.h = FNV_INIT;
        s.kn = 0;
        s.ef = (s.steps && in.exit_face) ? (int)in.exit_face[q] : MP_FACE_NONE;
        s.in_sink = 0;
        if (s.c >= 0 && (long long)s.c < f.ncell) {
            split_cell(f, s.c, s.k, s.i, s.j);
            s.h = (s.steps && in.hash) ? in.hash[q] : fnv_step(s.h, s.c);
            // a resumed particle may sit inside a sink cell it entered with
            // pass-through; a moving particle whose cell is not active under
            // this field (another flow period) stops there
            const int ib = __ldg(f.ibound + s.c);
            s.in_sink = ib == 2;
            if (s.st == MP_ST_ACTIVE) {
                if (ib == 0 || ib == -1) s.st = MP_ST_BOUNDARY;
                else if (ib == 2 && sink_stops(p, f.sinkfrac, s.c)) s.st = MP_ST_SINK;
            }
        } else {
            s.c = -1; s.i = s.j = s.k = 0;
            s.st = MP_ST_INVALID_RELEASE;
        }
        if (TS) {
            if (p.cont) {
                // output times up to the period start were written by the previous period
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= s.t) s.kn++;
            } else {
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= s.t) {
                    if (s.c >= 0) record(q, s.kn, s, gx(s), gy(s), gz(s), s.st);
                    else record(q, s.kn, s, CUDART_NAN, CUDART_NAN, CUDART_NAN, s.st);
                    s.kn++;
                }
            }
        }
        // a particle that starts at or after the stop time takes no step
        if (s.st == MP_ST_ACTIVE && s.t >= p.t_stop) s.st = MP_ST_TIME;
        s.tev = TS ? next_event(s) : p.t_stop;
    }

    // per-warp queue of deferred timeseries records (structure of arrays)
    struct RecQ {
        double p0[RQ_CAP], p1[RQ_CAP], p2[RQ_CAP], t[RQ_CAP];
        long long q[RQ_CAP];
        int c[RQ_CAP], i[RQ_CAP], j[RQ_CAP], k[RQ_CAP], kk[RQ_CAP], st[RQ_CAP], r[RQ_CAP];
    };

    __device__ __forceinline__ void rec_put(RecQ& Q, int slot, const State& s, long long q, int kk, int st) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        Q.r[slot] = s.r;
        Q.p0[slot] = s.x0; Q.p1[slot] = s.x1; Q.p2[slot] = s.x2;
        Q.t[slot] = s.t;   // tau = times[kk] - t is formed in rec_eval, where all 32 lanes take it
        Q.q[slot] = q;
        Q.c[slot] = s.c; Q.i[slot] = s.i; Q.j[slot] = s.j; Q.k[slot] = s.k;
        Q.kk[slot] = kk; Q.st[slot] = st;
    }

    // the position at tau after the step's start, by the motion formula on
    // every axis (the same operations as an endpoint stop at that time)
    __device__ __forceinline__ void rec_eval(const RecQ& Q, int slot) const
    {
        const Req& R = b.reqs[Q.r[slot]];
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        const int c = Q.c[slot], i = Q.i[slot], j = Q.j[slot], k = Q.k[slot];
        const double p0 = Q.p0[slot], p1 = Q.p1[slot], p2 = Q.p2[slot];
        const double tau = __ldg(o.times + Q.kk[slot]) - Q.t[slot];
        const double2* rp = reinterpret_cast<const double2*>(f.rec64 + c);
        const double2 r0 = __ldg(rp + 0), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2), r3 = __ldg(rp + 3),
                      r4 = __ldg(rp + 4);
        const double v1x = r0.x, Ax = r0.y, iAx = r1.x, v1y = r1.y, Ay = r2.x, iAy = r2.y;
        const double v1z = r3.x, Az = r3.y, iAz = r4.x;
        const double D0 = __ldg(f.delr + j), D1 = __ldg(f.delc + i), D2 = __ldg(f.dz + k);
        const double x = __ldg(f.xf + j) + move(Ax, iAx, D0, f64_vel(v1x, Ax, p0), p0, tau);
        const double y = __ldg(f.yf + i) + move(Ay, iAy, D1, f64_vel(v1y, Ay, p1), p1, tau);
        const double z = __ldg(f.zf + k) + move(Az, iAz, D2, f64_vel(v1z, Az, p2), p2, tau);
        store_record(o.ts + (long long)Q.kk[slot] * p.n + Q.q[slot], x, y, z, c, Q.st[slot]);
    }

    // One cell-step for every lane of the warp (warp-uniform call; lanes with
    // live == false only take part in the record queue).
    template <bool TS>
    __device__ __forceinline__ void step(long long q, State& s, bool live, RecQ& Q, int& qcount) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        enum { P_NONE, P_CROSS, P_TIME, P_NOEXIT, P_CAPTURE };
        int path = P_NONE;
        int m = 0;
        double v1x = 0, Ax = 0, v1y = 0, Ay = 0, v1z = 0, Az = 0, D0 = 1, D1 = 1, D2 = 1;
        double iAx = 0, iAy = 0, iAz = 0;
        double vp0 = 0, vp1 = 0, vp2 = 0, tmin = 0, t_end = 0;
        int f0 = 0, f1 = 0, f2 = 0, ax = -1;
        unsigned long long nb = 0;
        if (live) {
            if ((long long)s.steps >= p.max_steps) {
                s.st = MP_ST_STEP_CAP;
            } else if ((unsigned long long)s.c >= (unsigned long long)f.ncell) {
                atomicCAS(o.counters + COUNTER_ERR, 0ULL, (unsigned long long)q + 1ULL);
                s.st = MP_ST_INVALID_RELEASE;
            } else {
                const double2* rp = reinterpret_cast<const double2*>(f.rec64 + s.c);
                const double2 r0 = __ldg(rp + 0), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2), r3 = __ldg(rp + 3),
                              r4 = __ldg(rp + 4);
                const float4* rf = reinterpret_cast<const float4*>(rp + 5);
                const float4 g0 = __ldg(rf + 0), g1 = __ldg(rf + 1), g2 = __ldg(rf + 2);
                v1x = r0.x; Ax = r0.y; iAx = r1.x; v1y = r1.y; Ay = r2.x; iAy = r2.y;
                v1z = r3.x; Az = r3.y; iAz = r4.x;
                nb = (unsigned long long)__double_as_longlong(r4.y);
                const bool p2x = v2_pos(nb, 0), p2y = v2_pos(nb, 1), p2z = v2_pos(nb, 2);
                const bool n1x = v1_neg(nb, 0), n1y = v1_neg(nb, 1), n1z = v1_neg(nb, 2);
                D0 = __ldg(f.delr + s.j); D1 = __ldg(f.delc + s.i); D2 = __ldg(f.dz + s.k);
                vp0 = f64_vel(v1x, Ax, s.x0);
                vp1 = f64_vel(v1y, Ay, s.x1);
                vp2 = f64_vel(v1z, Az, s.x2);
                // reachable faces and FP32
                // estimates of the three exit times
                f0 = face_of(vp0, p2x, n1x);
                f1 = face_of(vp1, p2y, n1y);
                f2 = face_of(vp2, p2z, n1z);
                // estimates from FP32 distances to the reachable faces (the
                // FP64 distance is formed for the axes evaluated exactly)
                bool u0, u1, u2;
                const float e0 = estimate(f0, f32_face_dist(f0, D0, s.x0), vp0, g0.z, f0 > 0 ? g0.y : g0.x, u0);
                const float e1 = estimate(f1, f32_face_dist(f1, D1, s.x1), vp1, g1.y, f1 > 0 ? g1.x : g0.w, u1);
                const float e2 = estimate(f2, f32_face_dist(f2, D2, s.x2), vp2, g2.x, f2 > 0 ? g1.w : g1.z, u2);
                // candidates: every axis whose estimate is within 2^-10 of the
                // smallest (the estimates are within ~1.2e-4 of the exact times),
                // and every axis whose estimate cannot be trusted
                float em = CUDART_INF_F;
                int a0 = -1;
                if (f0 && !u0 && e0 < em) { em = e0; a0 = 0; }
                if (f1 && !u1 && e1 < em) { em = e1; a0 = 1; }
                if (f2 && !u2 && e2 < em) { em = e2; a0 = 2; }
                const float thr = em * (1.0f + 0.0009765625f);
                const unsigned cand = ((f0 && (u0 || e0 <= thr)) ? 1u : 0u) | ((f1 && (u1 || e1 <= thr)) ? 2u : 0u) |
                                      ((f2 && (u2 || e2 <= thr)) ? 4u : 0u);
                if (a0 < 0 && cand) a0 = __ffs(cand) - 1;
                tmin = CUDART_INF;
                if (a0 >= 0) {
                    // the exact FP64 exit time of the leading candidate (one
                    // evaluation per lane, uniform across the warp)
                    const int fa0 = sel3(a0, f0, f1, f2);
                    const double te = f64_exit_time_d(
                        sel3(a0, Ax, Ay, Az), sel3(a0, iAx, iAy, iAz),
                        f64_face_dist(fa0, sel3(a0, D0, D1, D2), sel3(a0, s.x0, s.x1, s.x2)),
                        sel3(a0, vp0, vp1, vp2), fa0);
                    // then the other candidates exactly (a close call; every
                    // reachable axis when the leading time is unusable): the
                    // smallest time wins, ties to the lower axis - the
                    // oracle's rule over all axes, since a non-candidate's
                    // exact time exceeds the leading one's
                    unsigned rest = cand & ~(1u << a0);
                    if (lt_inf(te)) {
                        tmin = te;
                        ax = a0;
                    } else {
                        rest = ((f0 ? 1u : 0u) | (f1 ? 2u : 0u) | (f2 ? 4u : 0u)) & ~(1u << a0);
                    }
                    while (rest) {
                        const int a = __ffs(rest) - 1;
                        rest &= rest - 1;
                        const int fa = sel3(a, f0, f1, f2);
                        const double t = f64_exit_time_d(
                            sel3(a, Ax, Ay, Az), sel3(a, iAx, iAy, iAz),
                            f64_face_dist(fa, sel3(a, D0, D1, D2), sel3(a, s.x0, s.x1, s.x2)),
                            sel3(a, vp0, vp1, vp2), fa);
                        if (t < tmin || (t == tmin && a < ax)) {
                            tmin = t;
                            ax = a;
                        }
                    }
                }
                s.steps++;
                t_end = s.t + tmin;
                if (ax < 0 && s.in_sink) path = P_CAPTURE;
                else if (ax < 0 && !(p.t_stop < CUDART_INF)) path = P_NOEXIT;
                else if (ax < 0 || ge_d(t_end, p.t_stop)) path = P_TIME;
                else path = P_CROSS;
                if (TS && path != P_CAPTURE && (ax < 0 || ge_d(t_end, s.tev))) {
                    const double t_rec = path == P_NOEXIT ? CUDART_INF : (path == P_TIME ? p.t_stop : t_end);
                    int kk = s.kn;
                    // (the comparison on the integer side, as in next_event)
                    while (kk < p.n_times && ge_d(t_rec, __ldg(o.times + kk))) kk++;
                    m = kk - s.kn;
                }
            }
        }
        if (TS && __any_sync(0xffffffffu, m > 0)) {
            rq_push(*this, Q, qcount, s, q, s.kn, m, path == P_NOEXIT ? MP_ST_NO_EXIT : MP_ST_ACTIVE);
            if (m) {
                s.kn += m;
                s.tev = next_event(s);
            }
        }
        if (path == P_NONE) return;
        if (path == P_CAPTURE) {
            s.st = MP_ST_SINK;
            return;
        }
        if (path == P_NOEXIT) {
            s.st = MP_ST_NO_EXIT;
            return;
        }
        if (path == P_TIME) {
            const double dt = p.t_stop - s.t;
            s.x0 = move(Ax, iAx, D0, vp0, s.x0, dt);
            s.x1 = move(Ay, iAy, D1, vp1, s.x1, dt);
            s.x2 = move(Az, iAz, D2, vp2, s.x2, dt);
            s.t = p.t_stop;
            s.st = MP_ST_TIME;
            return;
        }
        // displacement to the exit face: the two other axes move by the
        // analytic formula (selected into two slots, uniform across lanes),
        // the exit axis is put on its face
        const double dt = tmin;
        const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
        const double n1 = move(sel3(a1, Ax, Ay, Az), sel3(a1, iAx, iAy, iAz), sel3(a1, D0, D1, D2),
                               sel3(a1, vp0, vp1, vp2), sel3(a1, s.x0, s.x1, s.x2), dt);
        const double n2 = move(sel3(a2, Ax, Ay, Az), sel3(a2, iAx, iAy, iAz), sel3(a2, D0, D1, D2),
                               sel3(a2, vp0, vp1, vp2), sel3(a2, s.x0, s.x1, s.x2), dt);
        const int face = ax == 0 ? f0 : (ax == 1 ? f1 : f2);
        const double Dax = ax == 0 ? D0 : (ax == 1 ? D1 : D2);
        const double onface = face > 0 ? Dax : 0.0;
        s.x0 = ax == 0 ? onface : n1;
        s.x1 = ax == 1 ? onface : (ax == 0 ? n1 : n2);
        s.x2 = ax == 2 ? onface : n2;
        s.t = t_end;
        const int fidx = 2 * ax + (face > 0 ? 1 : 0);
        s.ef = fidx;
        const int cls = (int)((nb >> (2 * fidx)) & 3ULL);
        const int dj = ax == 0 ? face : 0, di = ax == 1 ? face : 0, dk = ax == 2 ? face : 0;
        if (cls != NB_ACTIVE &&
            !(cls == NB_SINK && !sink_stops(p, f.sinkfrac, s.c + dj + di * f.ncol + dk * f.ncol * f.nrow))) {
            s.st = cls == NB_OUTSIDE ? MP_ST_EXIT_DOMAIN : (cls == NB_BOUNDARY ? MP_ST_BOUNDARY : MP_ST_SINK);
            return;
        }
        s.in_sink = cls == NB_SINK;
        // hand over to the neighbour; the exit coordinate enters on the shared face
        s.j += dj;
        s.i += di;
        s.k += dk;
        s.c += dj + di * f.ncol + dk * f.ncol * f.nrow;
        // (the new cell's size along the exit axis, loaded by every lane:
        // one selected load instead of a branch on the direction)
        const double* sz = ax == 0 ? f.delr : (ax == 1 ? f.delc : f.dz);
        const int si = ax == 0 ? s.j : (ax == 1 ? s.i : s.k);
        const double entry = face < 0 ? __ldg(sz + si) : 0.0;
        s.x0 = ax == 0 ? entry : s.x0;
        s.x1 = ax == 1 ? entry : s.x1;
        s.x2 = ax == 2 ? entry : s.x2;
        s.h = fnv_step(s.h, s.c);
    }

    // the pathline point of the particle's current state
    __device__ __forceinline__ void path_point(const State& s, double& x, double& y, double& z, double& t) const
    {
        x = gx(s);
        y = gy(s);
        z = gz(s);
        t = s.t;
    }

    template <bool TS>
    __device__ __forceinline__ void finish(long long q, const State& s, unsigned long long* s_cnt) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        const bool ok = s.c >= 0;
        const unsigned base = in.steps ? in.steps[q] : 0u;   // read before the group update
        const double x = ok ? gx(s) : CUDART_NAN, y = ok ? gy(s) : CUDART_NAN, z = ok ? gz(s) : CUDART_NAN;
        o.cell[q] = s.c;
        o.x[q] = x; o.y[q] = y; o.z[q] = z;
        o.px[q] = s.x0; o.py[q] = s.x1; o.pz[q] = s.x2;
        o.t[q] = s.t;
        o.status[q] = (uint8_t)s.st;
        o.steps[q] = s.steps;
        o.exit_face[q] = (uint8_t)s.ef;
        o.hash[q] = s.h;
        if (p.update_group && ok) {
            in.cell[q] = s.c;
            in.px[q] = s.x0; in.py[q] = s.x1; in.pz[q] = s.x2;
            in.t[q] = s.t;
            in.status[q] = (uint8_t)((s.st == MP_ST_TIME || s.st == MP_ST_STEP_CAP) ? MP_ST_ACTIVE : s.st);
            if (in.steps) {
                in.steps[q] = s.steps;
                in.hash[q] = s.h;
                in.exit_face[q] = (uint8_t)s.ef;
            }
        }
        // steps taken in this launch; a particle paused at the end of a flow
        // period is counted by the period it ends in
        count_ended(b, s.r, s.steps - base, s.st, s_cnt, p.last || !(s.st == MP_ST_TIME || s.st == MP_ST_STEP_CAP));
    }
};

// The tracking kernels keep a launch's device-time window in its first
// request's counters; a batch's other requests get a copy.
__global__ void k_spread_window(const Req* reqs, int n)
{
    const unsigned long long* src = reqs[0].o.counters + COUNTER_T_BEGIN;
    const unsigned long long t0 = src[0], t1 = src[1];
    for (int i = 1 + (int)(blockIdx.x * blockDim.x + threadIdx.x); i < n; i += (int)(gridDim.x * blockDim.x)) {
        reqs[i].o.counters[COUNTER_T_BEGIN] = t0;
        reqs[i].o.counters[COUNTER_T_END] = t1;
    }
}

cudaError_t launch_spread_window(const Batch& b, cudaStream_t s)
{
    if (b.n_reqs <= 1 || b.n_total <= 0) return cudaSuccess;
    k_spread_window<<<1, 256, 0, s>>>(b.reqs, b.n_reqs);
    return cudaGetLastError();
}

cudaError_t launch_track_fp64(const DevField& f, const Batch& b, unsigned modes, int schedule, int block,
                              int blocks_per_sm_cap, cudaStream_t s)
{
    F64Engine e{f, b};
    return launch_tracking(e, modes, schedule, block, blocks_per_sm_cap, s);
}

}  // namespace mp

namespace mp {

// ---------------------------------------------------------------------------
// field validation: bit 1 non-finite flow, bit 2 porosity outside (0, 1] in
// an active or sink cell, bit 4 ibound outside {-1, 0, 1, 2}
// ---------------------------------------------------------------------------

__global__ void k_validate(const double* qx, long long nqx, const double* qy, long long nqy, const double* qz,
                           long long nqz, const double* por, const int8_t* ib, long long ncell, unsigned* flags)
{
    const long long total = nqx + nqy + nqz + ncell;
    unsigned bad = 0;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < total;
         u += (long long)gridDim.x * blockDim.x) {
        if (u < nqx) {
            if (!isfinite(qx[u])) bad |= 1u;
        } else if (u < nqx + nqy) {
            if (!isfinite(qy[u - nqx])) bad |= 1u;
        } else if (u < nqx + nqy + nqz) {
            if (!isfinite(qz[u - nqx - nqy])) bad |= 1u;
        } else {
            const long long c = u - nqx - nqy - nqz;
            const int8_t b = ib[c];
            if (b < -1 || b > 2) bad |= 4u;
            if (b == 1 || b == 2) {
                const double n = por[c];
                if (!(n > 0.0 && n <= 1.0)) bad |= 2u;
            }
        }
    }
    if (bad) atomicOr(flags, bad);
}

cudaError_t launch_validate(const double* qx, long long nqx, const double* qy, long long nqy, const double* qz,
                            long long nqz, const double* por, const int8_t* ib, long long ncell, unsigned* flags,
                            cudaStream_t s)
{
    k_validate<<<1024, 256, 0, s>>>(qx, nqx, qy, nqy, qz, nqz, por, ib, ncell, flags);
    return cudaGetLastError();
}

}  // namespace mp
