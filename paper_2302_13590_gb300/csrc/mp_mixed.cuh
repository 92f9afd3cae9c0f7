// mp_mixed.cuh - the mixed-precision tracking engine.
//
// Same method as the FP64 path (Pollock 1988: per-axis linear velocity,
// exit time (d / v_p) ln(1 + z) / z, analytic motion, smallest exit time
// wins, hand-over to the neighbour), evaluated in local fractions
// xi in [0, 1] of the cell with velocities u = v / D (1/s) in FP32:
//   u_p = u1 + A xi, A = u2 - u1, exit distance d = 1 - xi or -xi,
//   t_a = (d / u_p) g(z), z = A d / u_p, g(z) = ln(1 + z) / z,
//   xi(t) = xi + u_p t h(A t), h(w) = (e^w - 1) / w.
// g and h are evaluated both ways and selected (no divergent branch): their
// Taylor series near 0 (|z| < 1/8, |w| < 1/2; free of the 0/0 at 0),
// otherwise logf and expf (about 1 ulp, and free of the internal branches
// of log1pf and expm1f): g = ln(u) / (u - 1) with u = fl(1 + z), exact to a
// few ulp because the rounding of 1 + z cancels (Goldberg 1991), or
// ln(u_exit / u_p) / z for z < -1/2, where the ratio, not 1 + z, keeps full
// FP32 accuracy as u_exit -> 0.
//
// The cumulative travel time is carried as an unevaluated pair of FP32
// values (a double-float number, 48-bit significand): each step adds its
// FP32 step time with Knuth's error-free two-sum, and output times and the
// stop time are compared as pairs (the host splits them once per request).
// GB300 executes FP64 at 1/64 of the FP32 rate and output events occur in a
// different step on every lane, so FP64 arithmetic there would run in
// divergent branches; the pair keeps the time to ~1e-14 relative at FP32
// cost.  FP64 is used for the values written out: travel times and global
// positions.  Compiled with FMA contraction on (results are compared with the
// FP64 oracle within stated tolerances, not bit for bit).
//
// F64T = true gives the variant in which FP64 is kept for the cumulative
// travel time (one double, compared with the FP64 output and stop times)
// and for the near-zero branch of the exit time (log1p(z) / z evaluated in
// FP64 for |z| < 1/8); everything else is as above.  It exists to measure
// what the FP32 pair and the FP32 series cost in accuracy (mp_mixed_f64t.cu,
// MP_PREC_MIXED_F64T).
#pragma once
#include <cfloat>
#include <cmath>

#include "mp_internal.h"
#include "mp_sched.cuh"

namespace mp {

template <bool F64T>
struct MixEngine {
    // blocks of 256 threads to keep resident per SM: the kernels are issue
    // bound, and without a target the compiler gives the static endpoint
    // kernel fewer registers than it needs (spills); four blocks (at most 64
    // registers) fit both static kernels without spills
    static constexpr int min_blocks(bool dynamic, bool, bool pl) { return (!dynamic && !pl) ? 4 : 0; }
    DevField f;
    Batch b;

    struct State {
        int r;            // request of the particle within the launch
        int c, i, j, k;
        float x0, x1, x2;  // local fractions in [0, 1]
        float th, tl;  // travel time as an FP32 pair th + tl (F64T: unused)
        float eh, el;  // next output time or the stop time, whichever is first (as a pair)
        double t, e;   // F64T: travel time and next event in FP64
        unsigned steps;
        unsigned long long h;
        int kn;
        int st;
        int ef;
        int in_sink;      // the current cell is a sink entered with pass-through
    };

    // ---- double-float helpers (pairs with |lo| <= ulp(hi) / 2) ----
    // (nh, nl) = (th, tl) + dt, exact up to the final rounding of the low part
    __device__ __forceinline__ static void ff_add(float th, float tl, float dt, float& nh, float& nl)
    {
        const float sh = th + dt;
        const float bb = sh - th;
        const float lo = tl + ((th - (sh - bb)) + (dt - bb));
        nh = sh + lo;
        nl = lo - (nh - sh);
    }
    __device__ __forceinline__ static bool ff_ge(float ah, float al, float bh, float bl)
    {
        return ah > bh || (ah == bh && al >= bl);
    }
    // (a - b) as one FP32 value; a and b close, so the high parts cancel exactly
    __device__ __forceinline__ static float ff_diff(float ah, float al, float bh, float bl)
    {
        return (ah - bh) + (al - bl);
    }
    __device__ __forceinline__ static float2 time_pair(const DevOut& o, int kk)
    {
        return __ldg(o.times_ff + kk);
    }
    // the travel time as one FP64 value
    __device__ __forceinline__ static double time_of(const State& s)
    {
        if constexpr (F64T) return s.t;
        else return (double)s.th + (double)s.tl;
    }

    static constexpr float SMALL = 0.125f;

    // g(z) = ln(1 + z) / z, with 1 + z = u_exit / u_p: the series
    // sum_k (-z)^k / (k + 1) to degree 7 for |z| < 1/8; otherwise
    // ln(u) / (u - 1) with u = fl(1 + z), in which the rounding of 1 + z
    // cancels (Goldberg 1991), and for z < -1/2, where 1 + z itself
    // cancels, the logarithm of the ratio of the two stored velocities
    __device__ __forceinline__ static float g_log1p_over(float z, float ratio)
    {
        float ser;
        if constexpr (F64T) {
            // the near-zero branch in FP64: log1p(z) / z of the FP32 z (1 at z = 0)
            const double zd = (double)z;
            ser = (float)(zd == 0.0 ? 1.0 : log1p(zd) / zd);
        } else {
            ser = 1.0f + z * (-0.5f + z * (1.0f / 3.0f + z * (-0.25f + z * (0.2f + z * (-1.0f / 6.0f +
                                                                                  z * (1.0f / 7.0f + z * -0.125f))))));
        }
        const bool near_m1 = z < -0.5f;
        const float u = 1.0f + z;
        const float L = logf(near_m1 ? ratio : u);
        const float lg = __fdividef(L, near_m1 ? z : u - 1.0f);
        return fabsf(z) < SMALL ? ser : lg;
    }
    // h(w) = (e^w - 1) / w: sum_k w^k / (k + 1)! to degree 8 for |w| < 1/2
    // (truncation below 6e-10), otherwise the exponential (e^w - 1 then
    // loses at most a factor 2.5 to cancellation)
    __device__ __forceinline__ static float h_expm1_over(float w)
    {
        const float ser =
            1.0f + w * (0.5f + w * (1.0f / 6.0f + w * (1.0f / 24.0f + w * (1.0f / 120.0f + w * (1.0f / 720.0f +
                        w * (1.0f / 5040.0f + w * (1.0f / 40320.0f + w * (1.0f / 362880.0f))))))));
        const float ex = __fdividef(expf(w) - 1.0f, w);
        return fabsf(w) < 0.5f ? ser : ex;
    }

    template <class T>
    __device__ __forceinline__ static T sel3(int a, T x, T y, T z)
    {
        return a == 0 ? x : (a == 1 ? y : z);
    }

    // exit time along one axis in local units; branch-free around the
    // transcendental so that a warp's lanes stay converged (no-exit lanes
    // compute on harmless operands and select +inf)
    __device__ __forceinline__ static float exit_time(float u1, float u2, float A, float up, float xi, int& face)
    {
        const bool fw = up > 0.0f && u2 > 0.0f;
        const bool bw = up < 0.0f && u1 < 0.0f;
        face = fw ? 1 : (bw ? -1 : 0);
        const float d = fw ? 1.0f - xi : -xi;
        const float ue = fw ? u2 : u1;
        const float ups = face ? up : 1.0f;
        const float t1 = __fdividef(d, ups);
        const float g = g_log1p_over(A * t1, __fdividef(ue, ups));
        return face ? t1 * g : CUDART_INF_F;
    }

    __device__ __forceinline__ static float move(float A, float up, float xi, float dt)
    {
        const float s = up * dt;
        const float xn = fminf(fmaxf(xi + s * h_expm1_over(A * dt), 0.0f), 1.0f);
        return s == 0.0f ? xi : xn;
    }

    // global coordinate = face coordinate + fraction * cell size, rounded
    // step by step (no contraction) so endpoints and records agree exactly
    __device__ __forceinline__ double gx(const State& s, float xi) const
    {
        return __dadd_rn(__ldg(f.xf + s.j), __dmul_rn((double)xi, __ldg(f.delr + s.j)));
    }
    __device__ __forceinline__ double gy(const State& s, float xi) const
    {
        return __dadd_rn(__ldg(f.yf + s.i), __dmul_rn((double)xi, __ldg(f.delc + s.i)));
    }
    __device__ __forceinline__ double gz(const State& s, float xi) const
    {
        return __dadd_rn(__ldg(f.zf + s.k), __dmul_rn((double)xi, __ldg(f.dz + s.k)));
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

    __device__ __forceinline__ void final_pos(const State& s, double& x, double& y, double& z) const
    {
        if (s.c < 0) {
            x = y = z = CUDART_NAN;
            return;
        }
        x = gx(s, s.x0);
        y = gy(s, s.x1);
        z = gz(s, s.x2);
    }

    // next event as a pair: the next output time or the stop time
    __device__ __forceinline__ void next_event(State& s) const
    {
        const Req& R = b.reqs[s.r];
        const DevState& in = R.in;
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        (void)in; (void)o; (void)p;
        if constexpr (F64T) {
            double ev = p.t_stop;
            if (s.kn < p.n_times) ev = fmin(ev, __ldg(o.times + s.kn));
            s.e = ev;
            return;
        }
        float eh = p.tstop_hi, el = p.tstop_lo;
        if (s.kn < p.n_times) {
            const float2 tk = time_pair(o, s.kn);
            if (!ff_ge(tk.x, tk.y, eh, el)) { eh = tk.x; el = tk.y; }
        }
        s.eh = eh;
        s.el = el;
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
        const double t0 = in.t[q];
        // cell-steps, hash and last face carried by a resumed particle
        s.steps = in.steps ? in.steps[q] : 0u;
        s.h = FNV_INIT;
        s.kn = 0;
        s.ef = (s.steps && in.exit_face) ? (int)in.exit_face[q] : MP_FACE_NONE;
        s.in_sink = 0;
        if (s.c >= 0 && (long long)s.c < f.ncell) {
            split_cell(f, s.c, s.k, s.i, s.j);
            s.x0 = __fdiv_rn((float)in.px[q], (float)__ldg(f.delr + s.j));
            s.x1 = __fdiv_rn((float)in.py[q], (float)__ldg(f.delc + s.i));
            s.x2 = __fdiv_rn((float)in.pz[q], (float)__ldg(f.dz + s.k));
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
            s.x0 = s.x1 = s.x2 = 0.0f;
            s.st = MP_ST_INVALID_RELEASE;
        }
        if (TS) {
            if (p.cont) {
                // output times up to the period start were written by the previous period
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= t0) s.kn++;
            } else {
                while (s.kn < p.n_times && __ldg(o.times + s.kn) <= t0) {
                    if (s.c >= 0) record(q, s.kn, s, gx(s, s.x0), gy(s, s.x1), gz(s, s.x2), s.st);
                    else record(q, s.kn, s, CUDART_NAN, CUDART_NAN, CUDART_NAN, s.st);
                    s.kn++;
                }
            }
        }
        if (s.st == MP_ST_ACTIVE && t0 >= p.t_stop) s.st = MP_ST_TIME;
        s.th = (float)t0;
        s.tl = (float)(t0 - (double)s.th);
        if constexpr (F64T) s.t = t0;
        next_event(s);
    }

    // per-warp queue of deferred timeseries records (structure of arrays)
    struct RecQ {
        float x0[RQ_CAP], x1[RQ_CAP], x2[RQ_CAP], tau[RQ_CAP];
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
        Q.x0[slot] = s.x0; Q.x1[slot] = s.x1; Q.x2[slot] = s.x2;
        if constexpr (F64T) {
            Q.tau[slot] = (float)(__ldg(o.times + kk) - s.t);
        } else {
            const float2 tk = time_pair(o, kk);
            Q.tau[slot] = ff_diff(tk.x, tk.y, s.th, s.tl);
        }
        Q.q[slot] = q;
        Q.c[slot] = s.c; Q.i[slot] = s.i; Q.j[slot] = s.j; Q.k[slot] = s.k;
        Q.kk[slot] = kk; Q.st[slot] = st;
    }

    __device__ __forceinline__ void rec_eval(const RecQ& Q, int slot) const
    {
        const Req& R = b.reqs[Q.r[slot]];
        const DevOut& o = R.o;
        const TrackParams& p = R.p;
        State r;
        r.c = Q.c[slot]; r.i = Q.i[slot]; r.j = Q.j[slot]; r.k = Q.k[slot];
        const float tau = Q.tau[slot];
        const float4* rp = reinterpret_cast<const float4*>(f.rec32 + r.c);
        const float4 ra = __ldg(rp), rb = __ldg(rp + 1);
        const float Ax = ra.y - ra.x, Ay = ra.w - ra.z, Az = rb.y - rb.x;
        const float a0 = Q.x0[slot], a1 = Q.x1[slot], a2 = Q.x2[slot];
        const double x = gx(r, move(Ax, ra.x + Ax * a0, a0, tau));
        const double y = gy(r, move(Ay, ra.z + Ay * a1, a1, tau));
        const double z = gz(r, move(Az, rb.x + Az * a2, a2, tau));
        store_record(o.ts + (long long)Q.kk[slot] * p.n + Q.q[slot], x, y, z, r.c, Q.st[slot]);
    }

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
        float Ax = 0, Ay = 0, Az = 0, up0 = 0, up1 = 0, up2 = 0, tmin = 0, nh = 0, nl = 0;
        double tn = 0.0;   // F64T: the time at the end of the step
        (void)tn;
        bool ev = false;
        int f0 = 0, f1 = 0, f2 = 0, ax = -1;
        unsigned nb = 0;
        if (live) {
            if ((long long)s.steps >= p.max_steps) {
                s.st = MP_ST_STEP_CAP;
            } else if ((unsigned long long)s.c >= (unsigned long long)f.ncell) {
                atomicCAS(o.counters + COUNTER_ERR, 0ULL, (unsigned long long)q + 1ULL);
                s.st = MP_ST_INVALID_RELEASE;
            } else {
                const float4* rp = reinterpret_cast<const float4*>(f.rec32 + s.c);
                const float4 ra = __ldg(rp), rb = __ldg(rp + 1);
                const float u1x = ra.x, u2x = ra.y, u1y = ra.z, u2y = ra.w, u1z = rb.x, u2z = rb.y;
                nb = __float_as_uint(rb.z);
                Ax = u2x - u1x; Ay = u2y - u1y; Az = u2z - u1z;
                up0 = u1x + Ax * s.x0; up1 = u1y + Ay * s.x1; up2 = u1z + Az * s.x2;
                const float te0 = exit_time(u1x, u2x, Ax, up0, s.x0, f0);
                const float te1 = exit_time(u1y, u2y, Ay, up1, s.x1, f1);
                const float te2 = exit_time(u1z, u2z, Az, up2, s.x2, f2);
                tmin = CUDART_INF_F;
                if (f0 != 0 && te0 < tmin) { tmin = te0; ax = 0; }
                if (f1 != 0 && te1 < tmin) { tmin = te1; ax = 1; }
                if (f2 != 0 && te2 < tmin) { tmin = te2; ax = 2; }
                s.steps++;
                if constexpr (F64T) {
                    tn = s.t + (double)tmin;
                    ev = ax < 0 || tn >= s.e;
                } else {
                    ff_add(s.th, s.tl, tmin, nh, nl);
                    ev = ax < 0 || ff_ge(nh, nl, s.eh, s.el);
                }
                if (ev) {
                    bool past_stop;
                    if constexpr (F64T) past_stop = tn >= p.t_stop;
                    else past_stop = ff_ge(nh, nl, p.tstop_hi, p.tstop_lo);
                    if (ax < 0 && s.in_sink) path = P_CAPTURE;
                    else if (ax < 0 && !(p.t_stop < CUDART_INF)) path = P_NOEXIT;
                    else if (ax < 0 || past_stop) path = P_TIME;
                    else path = P_CROSS;
                    if (TS && path != P_CAPTURE) {
                        // output times inside this step: t_k <= end of step
                        int kk = s.kn;
                        if constexpr (F64T) {
                            const double r = path == P_NOEXIT ? CUDART_INF : (path == P_TIME ? p.t_stop : tn);
                            while (kk < p.n_times && __ldg(o.times + kk) <= r) kk++;
                        } else {
                            const float rh = path == P_NOEXIT ? CUDART_INF_F : (path == P_TIME ? p.tstop_hi : nh);
                            const float rl = path == P_NOEXIT ? 0.0f : (path == P_TIME ? p.tstop_lo : nl);
                            while (kk < p.n_times) {
                                const float2 tk = time_pair(o, kk);
                                if (!ff_ge(rh, rl, tk.x, tk.y)) break;
                                kk++;
                            }
                        }
                        m = kk - s.kn;
                    }
                } else {
                    path = P_CROSS;
                }
            }
        }
        if (TS && __any_sync(0xffffffffu, m > 0)) {
            rq_push(*this, Q, qcount, s, q, s.kn, m, path == P_NOEXIT ? MP_ST_NO_EXIT : MP_ST_ACTIVE);
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
            float dt;
            if constexpr (F64T) dt = (float)(p.t_stop - s.t);
            else dt = ff_diff(p.tstop_hi, p.tstop_lo, s.th, s.tl);
            s.x0 = move(Ax, up0, s.x0, dt);
            s.x1 = move(Ay, up1, s.x1, dt);
            s.x2 = move(Az, up2, s.x2, dt);
            s.th = p.tstop_hi;
            s.tl = p.tstop_lo;
            if constexpr (F64T) s.t = p.t_stop;
            s.st = MP_ST_TIME;
            return;
        }
        // the two other axes move by the analytic formula (two slots,
        // uniform across lanes), the exit axis is put on its face
        const float dt = tmin;
        const int a1 = ax == 0 ? 1 : 0, a2 = ax == 2 ? 1 : 2;
        const float n1 = move(sel3(a1, Ax, Ay, Az), sel3(a1, up0, up1, up2), sel3(a1, s.x0, s.x1, s.x2), dt);
        const float n2 = move(sel3(a2, Ax, Ay, Az), sel3(a2, up0, up1, up2), sel3(a2, s.x0, s.x1, s.x2), dt);
        const int face = ax == 0 ? f0 : (ax == 1 ? f1 : f2);
        const float onface = face > 0 ? 1.0f : 0.0f;
        s.x0 = ax == 0 ? onface : n1;
        s.x1 = ax == 1 ? onface : (ax == 0 ? n1 : n2);
        s.x2 = ax == 2 ? onface : n2;
        s.th = nh;
        s.tl = nl;
        if constexpr (F64T) s.t = tn;
        if (TS && m) {
            s.kn += m;
            next_event(s);
        }
        const int fidx = 2 * ax + (face > 0 ? 1 : 0);
        s.ef = fidx;
        const int cls = (int)((nb >> (2 * fidx)) & 3u);
        const int dj = ax == 0 ? face : 0, di = ax == 1 ? face : 0, dk = ax == 2 ? face : 0;
        if (cls != NB_ACTIVE &&
            !(cls == NB_SINK && !sink_stops(p, f.sinkfrac, s.c + dj + di * f.ncol + dk * f.ncol * f.nrow))) {
            s.st = cls == NB_OUTSIDE ? MP_ST_EXIT_DOMAIN : (cls == NB_BOUNDARY ? MP_ST_BOUNDARY : MP_ST_SINK);
            return;
        }
        s.in_sink = cls == NB_SINK;
        s.j += dj;
        s.i += di;
        s.k += dk;
        s.c += dj + di * f.ncol + dk * f.ncol * f.nrow;
        const float entry = face > 0 ? 0.0f : 1.0f;
        s.x0 = ax == 0 ? entry : s.x0;
        s.x1 = ax == 1 ? entry : s.x1;
        s.x2 = ax == 2 ? entry : s.x2;
        s.h = fnv_step(s.h, s.c);
    }

    // the pathline point of the particle's current state
    __device__ __forceinline__ void path_point(const State& s, double& x, double& y, double& z, double& t) const
    {
        x = gx(s, s.x0);
        y = gy(s, s.x1);
        z = gz(s, s.x2);
        t = time_of(s);
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
        double px = 0.0, py = 0.0, pz = 0.0, x = CUDART_NAN, y = CUDART_NAN, z = CUDART_NAN;
        if (ok) {
            px = __dmul_rn((double)s.x0, __ldg(f.delr + s.j));
            py = __dmul_rn((double)s.x1, __ldg(f.delc + s.i));
            pz = __dmul_rn((double)s.x2, __ldg(f.dz + s.k));
            x = gx(s, s.x0);
            y = gy(s, s.x1);
            z = gz(s, s.x2);
        }
        o.cell[q] = s.c;
        o.x[q] = x; o.y[q] = y; o.z[q] = z;
        o.px[q] = px; o.py[q] = py; o.pz[q] = pz;
        o.t[q] = time_of(s);
        o.status[q] = (uint8_t)s.st;
        o.steps[q] = s.steps;
        o.exit_face[q] = (uint8_t)s.ef;
        o.hash[q] = s.h;
        if (p.update_group && ok) {
            in.cell[q] = s.c;
            in.px[q] = px; in.py[q] = py; in.pz[q] = pz;
            in.t[q] = time_of(s);
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

}  // namespace mp
