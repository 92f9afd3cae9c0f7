// mp_usg.cu - FP64 tracking on rectangular unstructured (quadtree) grids.
//
// The paper's second test case also runs on a quadtree grid (TC2: refined
// near the boundary conditions); MODPATH moves particles there with the same
// Pollock displacement.  Cells are axis-aligned boxes whose faces may border
// several smaller cells.  Within a cell the velocity of each axis is linear
// between the face velocities, each from the face's total flow (its
// sub-faces summed in list order) over the cell's own face area; a particle
// that reaches a face enters the neighbour across the sub-face holding the
// exit point when that sub-face's flow runs with the crossing, else the
// nearest sub-face whose flow does (the point moves onto it), so opposing
// sub-face flows cannot bounce a particle back and forth.  Transverse
// offsets carry over through the difference of the two cells' origins.
//
// Compiled with -fmad=false: the same IEEE operations, in the same order, as
// the plain double-precision statement of the method; the cell-step itself
// (exit times, motion) is shared with the rectilinear FP64 engine.
#include <cfloat>
#include <cmath>

#include <cstddef>

#include "mp_internal.h"
#include "mp_sched.cuh"
#include "mp_f64math.cuh"

namespace mp {

// ---------------------------------------------------------------------------
// cell records and release
// ---------------------------------------------------------------------------

__device__ __forceinline__ double usg_face_flow(const DevUsg& u, long long c, int fi)
{
    const long long e0 = u.face_off[6 * c + fi], e1 = u.face_off[6 * c + fi + 1];
    if (e1 <= e0) return 0.0;
    double s = u.sub[e0].q;
    for (long long e = e0 + 1; e < e1; ++e) s += u.sub[e].q;
    return s;
}

// a cell's inflow and outflow from its face totals, face by face in the
// order x-, x+, y-, y+, z-, z+ (as the rectilinear grid's)
__device__ double2 usg_face_inout(const double q[6])
{
    double in = 0.0, out = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double q1 = q[2 * a], q2 = q[2 * a + 1];
        if (q1 > 0.0) in += q1; else out += -q1;
        if (q2 < 0.0) in += -q2; else out += q2;
    }
    return make_double2(in, out);
}

__global__ void k_build_usg(DevUsg u, UsgCell* out, UsgGeo* geo, double* sinkfrac, double2* inout,
                            const double* box, const double* por)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= u.ncell) return;
    const double* b = box + 6 * c;
    UsgGeo gm{};
    for (int a = 0; a < 3; ++a) { gm.o[a] = b[a]; gm.D[a] = b[3 + a]; }
    const int8_t ib = u.ibound[c];
    double v1[3] = {0.0, 0.0, 0.0}, v2[3] = {0.0, 0.0, 0.0};
    double sf = 0.0;
    double2 io = make_double2(0.0, 0.0);
    if (ib == 1 || ib == 2) {
        const double n = por[c];
        const double dx = b[3], dy = b[4], dzz = b[5];
        const double area[3] = {dy * dzz, dx * dzz, dx * dy};
        double q6[6];
        for (int fi = 0; fi < 6; ++fi) q6[fi] = usg_face_flow(u, c, fi);
        for (int a = 0; a < 3; ++a) {
            v1[a] = q6[2 * a] / (n * area[a]);
            v2[a] = q6[2 * a + 1] / (n * area[a]);
        }
        io = usg_face_inout(q6);
        if (ib == 2) sf = io.x > 0.0 ? (io.x - io.y) / io.x : 1.0;
    }
    sinkfrac[c] = sf;
    inout[c] = io;
    double A[3], iA[3];
    UsgCell r{};
    unsigned long long sg = 0;
    for (int a = 0; a < 3; ++a) {
        A[a] = (v2[a] - v1[a]) / b[3 + a];
        iA[a] = A[a] != 0.0 ? 1.0 / A[a] : 0.0;
        const unsigned long long bits4 = (v1[a] > 0.0 ? 1ULL : 0ULL) | (v1[a] < 0.0 ? 2ULL : 0ULL) |
                                         (v2[a] > 0.0 ? 4ULL : 0ULL) | (v2[a] < 0.0 ? 8ULL : 0ULL);
        sg |= bits4 << (4 * a);
    }
    r.v1x = v1[0]; r.Ax = A[0]; r.iAx = iA[0];
    r.v1y = v1[1]; r.Ay = A[1]; r.iAy = iA[1];
    r.v1z = v1[2]; r.Az = A[2]; r.iAz = iA[2];
    r.nb = sg;
    r.fv1x = (float)v1[0]; r.fv2x = (float)v2[0]; r.fAx = (float)A[0];
    r.fv1y = (float)v1[1]; r.fv2y = (float)v2[1]; r.fAy = (float)A[1];
    r.fv1z = (float)v1[2]; r.fv2z = (float)v2[2]; r.fAz = (float)A[2];
    out[c] = r;
    geo[c] = gm;
}

cudaError_t launch_build_usg(const DevUsg& u, UsgCell* cell, UsgGeo* geo, double* sinkfrac, double2* inout,
                             const double* box, const double* por, cudaStream_t s)
{
    if (u.ncell <= 0) return cudaSuccess;
    k_build_usg<<<(unsigned)((u.ncell + 255) / 256), 256, 0, s>>>(u, cell, geo, sinkfrac, inout, box, por);
    return cudaGetLastError();
}

__global__ void k_release_explicit_usg(DevUsg u, DevState st, long long n, const int32_t* cell, const double* local,
                                       const double* t0)
{
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const long long c = cell[q];
    st.t[q] = t0 ? t0[q] : 0.0;
    if (c < 0 || c >= u.ncell) {
        st.cell[q] = -1; st.px[q] = 0.0; st.py[q] = 0.0; st.pz[q] = 0.0;
        st.status[q] = MP_ST_INVALID_RELEASE;
        return;
    }
    const UsgGeo& r = u.geo[c];
    const double fx = fmin(fmax(local[3 * q], 0.0), 1.0);
    const double fy = fmin(fmax(local[3 * q + 1], 0.0), 1.0);
    const double fz = fmin(fmax(local[3 * q + 2], 0.0), 1.0);
    st.cell[q] = (int32_t)c;
    st.px[q] = fx * r.D[0]; st.py[q] = fy * r.D[1]; st.pz[q] = fz * r.D[2];
    const int8_t ib = u.ibound[c];
    st.status[q] = ib == 1 ? MP_ST_ACTIVE : (ib == 2 ? MP_ST_SINK : MP_ST_INVALID_RELEASE);
}

cudaError_t launch_release_explicit_usg(const DevUsg& u, const DevState& st, long long n, const int32_t* cell,
                                        const double* local, const double* t0, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_release_explicit_usg<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(u, st, n, cell, local, t0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// tracking engine
// ---------------------------------------------------------------------------

struct UsgEngine {
    static constexpr int min_blocks(bool, bool, bool) { return 0; }
    DevUsg u;
    Batch b;

    template <class T>
    __device__ __forceinline__ static T sel3(int a, T x, T y, T z)
    {
        return a == 0 ? x : (a == 1 ? y : z);
    }

    struct State {
        int r;
        int c;
        double x0, x1, x2;   // offsets (m) from the cell's low corner
        double t;
        unsigned steps;
        unsigned long long h;
        int kn;
        int st;
        int ef;
        int in_sink;
        double tev;
    };

    __device__ __forceinline__ double gx(const State& s) const { return __ldg(&u.geo[s.c].o[0]) + s.x0; }
    __device__ __forceinline__ double gy(const State& s) const { return __ldg(&u.geo[s.c].o[1]) + s.x1; }
    __device__ __forceinline__ double gz(const State& s) const { return __ldg(&u.geo[s.c].o[2]) + s.x2; }

    __device__ __forceinline__ void record(long long q, int kk, const State& s, double x, double y, double z,
                                           int st) const
    {
        const Req& R = b.reqs[s.r];
        store_record(R.o.ts + (long long)kk * R.p.n + q, x, y, z, s.c, st);
    }

    __device__ __forceinline__ void final_pos(const State& s, double& x, double& y, double& z) const
    {
        const bool ok = s.c >= 0;
        x = ok ? gx(s) : CUDART_NAN;
        y = ok ? gy(s) : CUDART_NAN;
        z = ok ? gz(s) : CUDART_NAN;
    }

    __device__ __forceinline__ double next_event(const State& s) const
    {
        const Req& R = b.reqs[s.r];
        const double tk = s.kn < R.p.n_times ? __ldg(R.o.times + s.kn) : CUDART_INF;
        return fmin(tk, R.p.t_stop);
    }

    template <bool TS>
    __device__ __forceinline__ void load(int r, long long q, State& s) const
    {
        s.r = r;
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        s.c = in.cell[q];
        s.st = in.status[q];
        if (p.cont && s.st != MP_ST_ACTIVE) {
            s.st = ST_SKIP;
            return;
        }
        s.x0 = in.px[q]; s.x1 = in.py[q]; s.x2 = in.pz[q];
        s.t = in.t[q];
        s.steps = in.steps ? in.steps[q] : 0u;
        s.h = FNV_INIT;
        s.kn = 0;
        s.ef = (s.steps && in.exit_face) ? (int)in.exit_face[q] : MP_FACE_NONE;
        s.in_sink = 0;
        if (s.c >= 0 && (long long)s.c < u.ncell) {
            s.h = (s.steps && in.hash) ? in.hash[q] : fnv_step(s.h, s.c);
            const int ib = __ldg(u.ibound + s.c);
            s.in_sink = ib == 2;
            if (s.st == MP_ST_ACTIVE) {
                if (ib == 0 || ib == -1) s.st = MP_ST_BOUNDARY;
                else if (ib == 2 && sink_stops(p, u.sinkfrac, s.c)) s.st = MP_ST_SINK;
            }
        } else {
            s.c = -1;
            s.st = MP_ST_INVALID_RELEASE;
        }
        if (TS) {
            if (p.cont) {
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= s.t) s.kn++;
            } else {
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= s.t) {
                    if (s.c >= 0) record(q, s.kn, s, gx(s), gy(s), gz(s), s.st);
                    else record(q, s.kn, s, CUDART_NAN, CUDART_NAN, CUDART_NAN, s.st);
                    s.kn++;
                }
            }
        }
        if (s.st == MP_ST_ACTIVE && s.t >= p.t_stop) s.st = MP_ST_TIME;
        s.tev = TS ? next_event(s) : p.t_stop;
    }

    struct RecQ {
        double p0[RQ_CAP], p1[RQ_CAP], p2[RQ_CAP], tau[RQ_CAP];
        long long q[RQ_CAP];
        int c[RQ_CAP], kk[RQ_CAP], st[RQ_CAP], r[RQ_CAP];
    };

    __device__ __forceinline__ void rec_put(RecQ& Q, int slot, const State& s, long long q, int kk, int st) const
    {
        const Req& R = b.reqs[s.r];
        Q.r[slot] = s.r;
        Q.p0[slot] = s.x0; Q.p1[slot] = s.x1; Q.p2[slot] = s.x2;
        Q.tau[slot] = __ldg(R.o.times + kk) - s.t;
        Q.q[slot] = q;
        Q.c[slot] = s.c;
        Q.kk[slot] = kk; Q.st[slot] = st;
    }

    __device__ __forceinline__ void rec_eval(const RecQ& Q, int slot) const
    {
        const Req& R = b.reqs[Q.r[slot]];
        const int c = Q.c[slot];
        const UsgCell& k = u.cell[c];
        const UsgGeo& g = u.geo[c];
        const double p0 = Q.p0[slot], p1 = Q.p1[slot], p2 = Q.p2[slot], tau = Q.tau[slot];
        const double x = __ldg(&g.o[0]) + f64_move(__ldg(&k.Ax), __ldg(&k.iAx), __ldg(&g.D[0]),
                                                   f64_vel(__ldg(&k.v1x), __ldg(&k.Ax), p0), p0, tau);
        const double y = __ldg(&g.o[1]) + f64_move(__ldg(&k.Ay), __ldg(&k.iAy), __ldg(&g.D[1]),
                                                   f64_vel(__ldg(&k.v1y), __ldg(&k.Ay), p1), p1, tau);
        const double z = __ldg(&g.o[2]) + f64_move(__ldg(&k.Az), __ldg(&k.iAz), __ldg(&g.D[2]),
                                                   f64_vel(__ldg(&k.v1z), __ldg(&k.Az), p2), p2, tau);
        store_record(R.o.ts + (long long)Q.kk[slot] * R.p.n + Q.q[slot], x, y, z, c, Q.st[slot]);
    }

    static_assert(offsetof(UsgSub, rect) % 16 == 0, "sub-face rectangles are read as 16-byte pairs");

    // the larger of a and b (non-NaN), chosen on the integer keys
    __device__ __forceinline__ static double kmax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }

    // L-infinity distance from (xa, xb) to a sub-face rectangle (0 inside):
    // four FP64 differences, the maxima taken on the ALU
    __device__ __forceinline__ static double rect_dist(const UsgSub& e, double xa, double xb)
    {
        const double m = kmax(kmax(e.rect[0] - xa, xa - e.rect[1]), kmax(e.rect[2] - xb, xb - e.rect[3]));
        return lt0(m) ? 0.0 : m;
    }

    // the flow of sub-face e runs with a crossing to `side` (q * side > 0;
    // face flows are finite)
    __device__ __forceinline__ bool with_flow(long long e, int side) const
    {
        const double qe = __ldg(&u.sub[e].q);
        return side > 0 ? gt0(qe) : lt0(qe);
    }

    // the neighbour across face (ax, side) at the exit point (xa, xb) =
    // cell origin + offset on the two other axes: the first sub-face holding
    // it (else the nearest, first on ties) if its flow runs with the
    // crossing, else the nearest one whose flow does, the point moved onto
    // it (mva / mvb: that coordinate changed); -1: no sub-face (outside).  A
    // face with one sub-face hands over to its neighbour either way, so
    // neither the exit point nor a distance is formed there.  Whether a
    // rectangle holds the point is decided on the integer keys of the
    // coordinates (the ALU pipe): only a lane crossing a refined face runs
    // this, so FP64 work here would hold the whole warp's FP64 pipe for a
    // few lanes; distances are formed only when no rectangle holds it.
    __device__ __forceinline__ int across(int c, int ax, int side, double oa_, double pa_, double ob_, double pb_,
                                          double& xa, double& xb, bool& mva, bool& mvb) const
    {
        mva = mvb = false;
        const int fi = 2 * ax + (side > 0 ? 1 : 0);
        const long long e0 = __ldg(u.face_off + 6LL * c + fi), e1 = __ldg(u.face_off + 6LL * c + fi + 1);
        if (e1 <= e0) return -1;
        if (e1 - e0 == 1) return __ldg(&u.sub[e0].nbr);
        xa = oa_ + pa_;
        xb = ob_ + pb_;
        const long long ka = dkey(xa), kb = dkey(xb);
        long long best = -1;
        for (long long e = e0; e < e1; ++e) {
            const double2* r = reinterpret_cast<const double2*>(u.sub[e].rect);
            const double2 ra = __ldg(r), rb = __ldg(r + 1);
            if (dkey(ra.x) <= ka && ka <= dkey(ra.y) && dkey(rb.x) <= kb && kb <= dkey(rb.y)) {
                best = e;
                break;
            }
        }
        if (best < 0) {
            best = e0;
            double bd = CUDART_INF;
            for (long long e = e0; e < e1; ++e) {
                const double d = rect_dist(u.sub[e], xa, xb);
                if (dkey(d) < dkey(bd)) { bd = d; best = e; }
            }
        }
        if (with_flow(best, side)) return u.sub[best].nbr;
        long long alt = -1;
        double ad = CUDART_INF;
        for (long long e = e0; e < e1; ++e) {
            if (!with_flow(e, side)) continue;
            const double d = rect_dist(u.sub[e], xa, xb);
            if (dkey(d) < dkey(ad)) { ad = d; alt = e; }
        }
        if (alt < 0) return u.sub[best].nbr;
        const UsgSub& e = u.sub[alt];
        const double na = fmin(fmax(xa, e.rect[0]), e.rect[1]);
        const double nb = fmin(fmax(xb, e.rect[2]), e.rect[3]);
        mva = dkey(na) != dkey(xa);
        mvb = dkey(nb) != dkey(xb);
        xa = na;
        xb = nb;
        return e.nbr;
    }

    template <bool TS>
    __device__ __forceinline__ void step(long long q, State& s, bool live, RecQ& Q, int& qcount) const
    {
        const Req& R = b.reqs[s.r];
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        enum { P_NONE, P_CROSS, P_TIME, P_NOEXIT, P_CAPTURE };
        int path = P_NONE;
        int m = 0;
        double v1[3] = {0, 0, 0}, A[3] = {0, 0, 0}, iA[3] = {0, 0, 0}, D[3] = {1, 1, 1}, org[3] = {0, 0, 0};
        double vp[3] = {0, 0, 0}, tmin = 0, t_end = 0;
        int fc[3] = {0, 0, 0}, ax = -1;
        if (live) {
            if ((long long)s.steps >= p.max_steps) {
                s.st = MP_ST_STEP_CAP;
            } else if ((unsigned long long)s.c >= (unsigned long long)u.ncell) {
                atomicCAS(o.counters + COUNTER_ERR, 0ULL, (unsigned long long)q + 1ULL);
                s.st = MP_ST_INVALID_RELEASE;
            } else {
                const double2* rp = reinterpret_cast<const double2*>(u.cell + s.c);
                const double2 r0 = __ldg(rp + 0), r1 = __ldg(rp + 1), r2 = __ldg(rp + 2), r3 = __ldg(rp + 3),
                              r4 = __ldg(rp + 4);
                const float4* rf = reinterpret_cast<const float4*>(rp + 5);
                const float4 g0 = __ldg(rf + 0), g1 = __ldg(rf + 1), g2 = __ldg(rf + 2);
                const double2* gp = reinterpret_cast<const double2*>(u.geo + s.c);
                const double2 q0 = __ldg(gp + 0), q1 = __ldg(gp + 1), q2 = __ldg(gp + 2);
                v1[0] = r0.x; A[0] = r0.y; iA[0] = r1.x; v1[1] = r1.y; A[1] = r2.x; iA[1] = r2.y;
                v1[2] = r3.x; A[2] = r3.y; iA[2] = r4.x;
                const unsigned long long sg = (unsigned long long)__double_as_longlong(r4.y);
                org[0] = q0.x; org[1] = q0.y; org[2] = q1.x; D[0] = q1.y; D[1] = q2.x; D[2] = q2.y;
                const double pp[3] = {s.x0, s.x1, s.x2};
                bool p2[3], n1[3];
                float dd[3];
                #pragma unroll
                for (int a = 0; a < 3; ++a) {
                    vp[a] = f64_vel(v1[a], A[a], pp[a]);
                    p2[a] = (sg >> (4 * a + 2)) & 1ULL;
                    n1[a] = (sg >> (4 * a + 1)) & 1ULL;
                    fc[a] = f64_face(vp[a], p2[a], n1[a]);
                    dd[a] = f32_face_dist(fc[a], D[a], pp[a]);
                }
                // FP32 estimates of the three exit times (from FP32 face
                // distances); the exact FP64 time of the leading one, and of
                // every axis within 2^-10 of it or with an untrusted
                // estimate (the same exit axis and time as evaluating all
                // three exactly)
                bool u0, u1, u2;
                const float e0 = f32_estimate_f(fc[0], dd[0], vp[0], g0.z,
                                                fc[0] > 0 ? g0.y : g0.x, u0);
                const float e1 = f32_estimate_f(fc[1], dd[1], vp[1], g1.y,
                                                fc[1] > 0 ? g1.x : g0.w, u1);
                const float e2 = f32_estimate_f(fc[2], dd[2], vp[2], g2.x,
                                                fc[2] > 0 ? g1.w : g1.z, u2);
                float em = CUDART_INF_F;
                int a0 = -1;
                if (fc[0] && !u0 && e0 < em) { em = e0; a0 = 0; }
                if (fc[1] && !u1 && e1 < em) { em = e1; a0 = 1; }
                if (fc[2] && !u2 && e2 < em) { em = e2; a0 = 2; }
                const float thr = em * (1.0f + 0.0009765625f);
                const unsigned cand = ((fc[0] && (u0 || e0 <= thr)) ? 1u : 0u) | ((fc[1] && (u1 || e1 <= thr)) ? 2u : 0u) |
                                      ((fc[2] && (u2 || e2 <= thr)) ? 4u : 0u);
                if (a0 < 0 && cand) a0 = __ffs(cand) - 1;
                tmin = CUDART_INF;
                if (a0 >= 0) {
                    const int fa0 = sel3(a0, fc[0], fc[1], fc[2]);
                    const double te = f64_exit_time_d(
                        sel3(a0, A[0], A[1], A[2]), sel3(a0, iA[0], iA[1], iA[2]),
                        f64_face_dist(fa0, sel3(a0, D[0], D[1], D[2]), sel3(a0, pp[0], pp[1], pp[2])),
                        sel3(a0, vp[0], vp[1], vp[2]), fa0);
                    // the other candidates (every reachable axis when the
                    // leading time is unusable): smallest wins, ties to the
                    // lower axis
                    unsigned rest = cand & ~(1u << a0);
                    if (lt_inf(te)) {
                        tmin = te;
                        ax = a0;
                    } else {
                        rest = ((fc[0] ? 1u : 0u) | (fc[1] ? 2u : 0u) | (fc[2] ? 4u : 0u)) & ~(1u << a0);
                    }
                    while (rest) {
                        const int a = __ffs(rest) - 1;
                        rest &= rest - 1;
                        const int fa = sel3(a, fc[0], fc[1], fc[2]);
                        const double t = f64_exit_time_d(
                            sel3(a, A[0], A[1], A[2]), sel3(a, iA[0], iA[1], iA[2]),
                            f64_face_dist(fa, sel3(a, D[0], D[1], D[2]), sel3(a, pp[0], pp[1], pp[2])),
                            sel3(a, vp[0], vp[1], vp[2]), fa);
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
                    while (kk < p.n_times && __ldg(o.times + kk) <= t_rec) kk++;
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
        double pp[3] = {s.x0, s.x1, s.x2};
        if (path == P_TIME) {
            const double dt = p.t_stop - s.t;
            #pragma unroll
            for (int a = 0; a < 3; ++a) pp[a] = f64_move(A[a], iA[a], D[a], vp[a], pp[a], dt);
            s.x0 = pp[0]; s.x1 = pp[1]; s.x2 = pp[2];
            s.t = p.t_stop;
            s.st = MP_ST_TIME;
            return;
        }
        // the two other axes move (two slots, uniform across lanes), the exit
        // axis is put on its face
        const double dt = tmin;
        const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
        const double n1v = f64_move(sel3(a1, A[0], A[1], A[2]), sel3(a1, iA[0], iA[1], iA[2]),
                                    sel3(a1, D[0], D[1], D[2]), sel3(a1, vp[0], vp[1], vp[2]),
                                    sel3(a1, pp[0], pp[1], pp[2]), dt);
        const double n2v = f64_move(sel3(a2, A[0], A[1], A[2]), sel3(a2, iA[0], iA[1], iA[2]),
                                    sel3(a2, D[0], D[1], D[2]), sel3(a2, vp[0], vp[1], vp[2]),
                                    sel3(a2, pp[0], pp[1], pp[2]), dt);
        const int side = sel3(ax, fc[0], fc[1], fc[2]);
        const double pf = side > 0 ? sel3(ax, D[0], D[1], D[2]) : 0.0;
        pp[0] = ax == 0 ? pf : n1v;
        pp[1] = ax == 1 ? pf : (ax == 0 ? n1v : n2v);
        pp[2] = ax == 2 ? pf : n2v;
        s.x0 = pp[0]; s.x1 = pp[1]; s.x2 = pp[2];
        s.t = t_end;
        s.ef = 2 * ax + (side > 0 ? 1 : 0);
        // hand over at the exit point
        const int oa = ax == 0 ? 1 : 0, ob = ax == 2 ? 1 : 2;
        double xa = 0.0, xb = 0.0;
        bool mva, mvb;
        const int nc = across(s.c, ax, side, sel3(oa, org[0], org[1], org[2]), sel3(oa, pp[0], pp[1], pp[2]),
                              sel3(ob, org[0], org[1], org[2]), sel3(ob, pp[0], pp[1], pp[2]), xa, xb, mva, mvb);
        if (nc < 0) {
            s.st = MP_ST_EXIT_DOMAIN;
            return;
        }
        const int ib = __ldg(u.ibound + nc);
        if (ib == 0 || ib == -1) {
            s.st = MP_ST_BOUNDARY;
            return;
        }
        if (ib == 2 && sink_stops(p, u.sinkfrac, nc)) {
            s.st = MP_ST_SINK;
            return;
        }
        s.in_sink = ib == 2;
        const UsgGeo& n = u.geo[nc];
        double on[3], Dn[3];
        #pragma unroll
        for (int a = 0; a < 3; ++a) { on[a] = __ldg(&n.o[a]); Dn[a] = __ldg(&n.D[a]); }
        // the other two axes keep their global coordinate, p + (o - o'); a
        // hand-over that moved the point enters at the moved point x, as
        // x + (-o') (the rounding of x - o').  One form with operands chosen
        // on the ALU, so every lane runs the same two additions per axis.
        double pt[2];
        #pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int a = t == 0 ? oa : ob;
            const bool mv = t == 0 ? mva : mvb;
            const double on_a = sel3(a, on[0], on[1], on[2]);
            const double dor = sel3(a, org[0], org[1], org[2]) - on_a;
            const double X = mv ? (t == 0 ? xa : xb) : sel3(a, pp[0], pp[1], pp[2]);
            double pa = X + (mv ? neg(on_a) : dor);
            const double Da = sel3(a, Dn[0], Dn[1], Dn[2]);
            pa = lt0(pa) ? 0.0 : pa;
            pt[t] = gt_pos(pa, Da) ? Da : pa;
        }
        const double pe = side > 0 ? 0.0 : sel3(ax, Dn[0], Dn[1], Dn[2]);
        s.x0 = ax == 0 ? pe : pt[0];
        s.x1 = ax == 1 ? pe : (ax == 0 ? pt[0] : pt[1]);
        s.x2 = ax == 2 ? pe : pt[1];
        s.c = nc;
        s.h = fnv_step(s.h, s.c);
    }

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
        const bool ok = s.c >= 0;
        const unsigned base = in.steps ? in.steps[q] : 0u;
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
        count_ended(b, s.r, s.steps - base, s.st, s_cnt, p.last || !(s.st == MP_ST_TIME || s.st == MP_ST_STEP_CAP));
    }
};

cudaError_t launch_track_usg(const DevUsg& u, const Batch& b, unsigned modes, int schedule, int block,
                             int blocks_per_sm_cap, cudaStream_t s)
{
    UsgEngine e{u, b};
    return launch_tracking(e, modes, schedule, block, blocks_per_sm_cap, s);
}

}  // namespace mp
