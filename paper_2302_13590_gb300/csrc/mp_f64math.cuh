// mp_f64math.cuh - the FP64 arithmetic of a Pollock cell-step, shared by the
// rectilinear and the unstructured FP64 engines.  Every translation unit
// that includes it is compiled with -fmad=false: each multiply and add
// rounds on its own, in the order written, the operations of the plain
// double-precision statement of the method.
#pragma once

#include <math_constants.h>

#include "mp_f64_tables.h"

namespace mp {

// ---------------------------------------------------------------------------
// Exact tests and scalings on the bits of a double.  GB300 runs FP64 at 1/64
// of the FP32 rate and the FP64 kernel is bound by its FP64 pipe, so sign,
// zero and order tests with a known sign, frexp and ldexp are done as
// integer operations on the representation (the ALU pipe is idle); each
// gives exactly the IEEE result for the non-NaN operands the path produces.
// ---------------------------------------------------------------------------

// The representation of v, opaque to the optimiser (an empty asm): without
// it the compiler folds tests such as (bits << 1) == 0 back into FP64
// compares, which run on the FP64 pipe.
__device__ __forceinline__ long long bits(double v)
{
    long long b = __double_as_longlong(v);
    asm("" : "+l"(b));
    return b;
}
// v > 0
__device__ __forceinline__ bool gt0(double v) { return bits(v) > 0LL; }
// v < 0 (-0 is not)
__device__ __forceinline__ bool lt0(double v)
{
    return (unsigned long long)bits(v) > 0x8000000000000000ULL;
}
// v == 0 (either sign)
__device__ __forceinline__ bool eq0(double v) { return (bits(v) << 1) == 0LL; }
// a > b for b > 0
__device__ __forceinline__ bool gt_pos(double a, double b) { return bits(a) > bits(b); }
// |a| < b for b > 0
__device__ __forceinline__ bool abs_lt(double a, double b) { return (bits(a) & 0x7fffffffffffffffLL) < bits(b); }
__device__ __forceinline__ bool is_nan(double v)
{
    return (bits(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

// an integer key whose order is the IEEE order of non-NaN doubles (-0 and
// +0 share key 0): a >= b exactly when dkey(a) >= dkey(b)
__device__ __forceinline__ long long dkey(double v)
{
    const long long b = bits(v);
    return b >= 0LL ? b : -(b & 0x7fffffffffffffffLL);
}
// a >= b for non-NaN a, b
__device__ __forceinline__ bool ge_d(double a, double b) { return dkey(a) >= dkey(b); }
// v < +inf (false for +inf and NaN)
__device__ __forceinline__ bool lt_inf(double v)
{
    return (bits(v) & 0x7fffffffffffffffLL) < 0x7ff0000000000000LL || bits(v) == (long long)0xfff0000000000000ULL;
}

// -v (the sign bit flipped, as IEEE negation)
__device__ __forceinline__ double neg(double v)
{
    return __longlong_as_double(bits(v) ^ (long long)0x8000000000000000ULL);
}

// The helpers below compute every case and select (no branch): the FP64
// kernels' lanes then stay converged through them.

// frexp of a positive normal finite u: u = m 2^e with m in [1/2, 1)
__device__ __forceinline__ double frexp_normal(double u, int& e)
{
    const long long b = bits(u);
    e = (int)(b >> 52) - 1022;
    return __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3fe0000000000000LL);
}

// (double)e for |e| < 2^30, exactly
__device__ __forceinline__ double i2d_exact(int e)
{
    const unsigned long long sgn = e < 0 ? 0x8000000000000000ULL : 0ULL;
    const unsigned a = (unsigned)(e < 0 ? -e : e);
    const int msb = 31 - __clz(a | 1u);
    const unsigned long long mant = ((unsigned long long)a << (52 - msb)) & 0x000fffffffffffffULL;
    const unsigned long long r = sgn | ((unsigned long long)(1023 + msb) << 52) | mant;
    return __longlong_as_double(a == 0u ? 0LL : (long long)r);
}

// 2^k as ldexp(1, k) gives it, k in [-2000, 2000]
__device__ __forceinline__ double pow2i(int k)
{
    const unsigned long long nrm = (unsigned long long)(k + 1023) << 52;        // -1022 <= k <= 1023
    const unsigned long long sub = 1ULL << ((unsigned)(k + 1074) & 63u);        // -1074 <= k < -1022
    unsigned long long r = k >= -1022 ? nrm : (k >= -1074 ? sub : 0ULL);
    r = k >= 1024 ? 0x7ff0000000000000ULL : r;
    return __longlong_as_double((long long)r);
}

// FP64 -> FP32 by truncating the significand on the ALU pipe (the FP64
// pipe, the binding unit of the FP64 kernels, is spared the conversion):
// relative error below 2^-23; magnitudes below the FP32 normal range give
// 0, above it (and infinities, NaN) give infinity, with the sign.
__device__ __forceinline__ float f32_trunc(double x)
{
    const long long b = bits(x);
    const unsigned s = (unsigned)((unsigned long long)b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned nrm = s | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
    return __uint_as_float(e < -126 ? s : (e > 127 ? (s | 0x7f800000u) : nrm));
}

// (float)u rounded to nearest even, for u >= 2^-126 (the values 1 + x
// takes in log1p are >= 2^-53), on the ALU pipe; above the FP32 range:
// infinity, as the conversion gives
__device__ __forceinline__ float f32_rn_pos(double u)
{
    const long long b = bits(u);
    const int e = (int)(b >> 52) - 1023;
    unsigned fb = ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffff);
    const unsigned rem = (unsigned)(b & 0x1fffffff);
    fb += (rem > 0x10000000u || (rem == 0x10000000u && (fb & 1u))) ? 1u : 0u;
    return __uint_as_float(e > 127 ? 0x7f800000u : fb);
}

// (double)f for f >= 0 (zero, subnormal, normal, infinity: on the ALU pipe;
// a subnormal's fraction is normalised by its leading-zero count)
__device__ __forceinline__ double f2d_pos(float f)
{
    const unsigned fb = __float_as_uint(f);
    const unsigned fe = fb >> 23;
    const unsigned fm = fb & 0x7fffffu;
    const int sh = __clz(fm | 1u) - 8;   // brings a subnormal's leading 1 to bit 23
    const unsigned long long sub = ((unsigned long long)(897 - sh) << 52) |
                                   ((unsigned long long)((fm << sh) & 0x7fffffu) << 29);
    const unsigned long long nrm = ((unsigned long long)(fe + 896u) << 52) | ((unsigned long long)fm << 29);
    unsigned long long r = fe == 0u ? (fm == 0u ? 0ULL : sub) : nrm;
    r = fe == 255u ? 0x7ff0000000000000ULL : r;
    return __longlong_as_double((long long)r);
}

// (double)f for a normal f of either sign (no branch: the callers' values
// are normal by construction)
__device__ __forceinline__ double f2d_normal(float f)
{
    const unsigned fb = __float_as_uint(f);
    return __longlong_as_double(((long long)(fb >> 31) << 63) | ((long long)(((fb >> 23) & 0xffu) + 896u) << 52) |
                                ((long long)(fb & 0x7fffffu) << 29));
}

// d / v as d times 1 / v: the IEEE FP32 reciprocal y0 of the truncated v
// (relative error below 1.8e-7), then one third-order step
// y = y0 + y0 (e + e^2) with e = 1 - v y0 in one fma (rounded by less
// than 2^-75), which leaves e^3 < 2^-67 and the roundings, so 1 / v
// within about half an ulp and the quotient within about one (three fmas
// where two Newton steps take four).  |v| outside [2^-120, 2^121) (and 0,
// infinity, NaN) takes the IEEE division.
static __device__ __noinline__ double div_ieee(double a, double b) { return a / b; }

__device__ __forceinline__ double f64_div(double d, double v)
{
    const int e = (int)((bits(v) >> 52) & 0x7ff) - 1023;
    if (e < -120 || e > 120) return div_ieee(d, v);
    const double y0 = f2d_normal(__frcp_rn(f32_trunc(v)));   // |1 / v| in (2^-121, 2^120]: normal
    const double e0 = fma(-v, y0, 1.0);
    const double y1 = fma(y0, fma(e0, e0, e0), y0);
    return d * y1;
}

// ---------------------------------------------------------------------------
// log1p and expm1 by argument reduction, a table and a short series, with
// IEEE additions, multiplications and explicit fused multiply-adds in a
// fixed order (no implicit contraction: this file is built with
// -fmad=false), exact bit operations on the ALU pipe, one FP32 reciprocal
// and FP32 products, so that the FP64 path produces the same bits as any
// other evaluation of the same steps on the host.  Exit-axis choices near a
// tie then agree exactly, which library functions with different last-bit
// rounding cannot guarantee on ill-conditioned fields.  The method is
// Tang's table-driven one (P. T. P. Tang, "Table-driven implementation of
// the exponential function in IEEE floating-point arithmetic", ACM TOMS
// 15(2), 1989; "Table-driven implementation of the logarithm function in
// IEEE floating-point arithmetic", ACM TOMS 16(4), 1990), with tables and
// series lengths of this file's own choosing.  The tables
// (mp_f64_tables.h) hold correctly rounded constants.
//   log1p(x): u = 1 + x; u = m 2^e with m in [1/sqrt2, sqrt2); the bucket
//     of m (exponent and top 8 fraction bits) gives R ~ 1/m with 8
//     significant bits and -ln R = Lh + Ll.  For e in [-2, 3] (u in
//     [1/(4 sqrt2), 8 sqrt2): all but a few in ten thousand exit times,
//     also on strongly heterogeneous fields with wells) a
//     table row per (e, bucket) holds e ln2_hi + Lh (exact), e ln2_lo + Ll
//     rounded, R' = R 2^-e and R' - 1 (exact), and r = (1 + x) R' - 1 =
//     x R' + (R' - 1) is one fma on x itself, so the rounding of 1 + x never
//     enters; otherwise (out of line) r = m R - 1 exactly and the rounding
//     error c of 1 + x (two-sum) is added as c times the FP32 reciprocal of
//     u.  ln(1 + r) by its series to r^8 (|r| < 0.006), the factor of r^5
//     in FP32 on the truncated r; result (e ln2_hi + Lh) +
//     (ln(1 + r) + (e ln2_lo + Ll)).  u = +inf -> +inf, u = 0 -> -inf,
//     NaN -> NaN.
//   expm1(w): |w| limited to 800; k = nearest integer to w 256/ln2 in FP32
//     on the truncated w; j = k mod 256, m = (k - j) / 256;
//     r = w - k ln2_hi/256 (exact); expm1(r) by its series to r^5
//     (|r| < 0.0016), the factor of r^4 in FP32 on the truncated r.  For
//     m in [-2, 1] (|w| below about 2 ln2: all but a few in a thousand
//     motions, also on strongly heterogeneous fields with wells) expm1(w) =
//     A em + B in one fma, A = e^(k ln2_hi/256) and B = A - 1 rounded from
//     a table (the low part of k ln2/256 is in the table); otherwise (out
//     of line) r -= k ln2_lo/256, 2^(j/256) = Th + Tl, S = Th expm1(r) + Tl,
//     expm1(w) = (2^m Th - 1) + 2^m S ((Th + S) 2^(m-1023) 2^1023 when
//     2^m is not finite).  About 9 and 6 FP64 operations.
// ---------------------------------------------------------------------------

// ln(1 + r) by its series to r^8; the tail 1/5 - r/6 + r^2/7 - r^3/8 in
// FP32: it enters scaled by r^5, below 2.6e-10 of the result, so its FP32
// error stays below 0.15 ulp (and the FP64 pipe is spared three fmas)
__device__ __forceinline__ double log1p_series(double r)
{
    const double r2 = r * r;
    const float rf = f32_trunc(r);
    float pf = __fmaf_rn(-0x1.0p-3f, rf, 0x1.24924ap-3f);   // -1/8, 1/7
    pf = __fmaf_rn(pf, rf, -0x1.555556p-3f);                // -1/6
    pf = __fmaf_rn(pf, rf, 0x1.99999ap-3f);                 // 1/5
    double q = fma(r, f2d_normal(pf), -0.25);   // pf near 1/5: normal
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    return fma(r2, q, r);
}

// log1p for exponents e outside the table rows (rare; out of line, and a
// side effect keeps the call from being evaluated speculatively):
// r = m R - 1 exactly and the two-sum error c of u = 1 + x as c / u
static __device__ __noinline__ double log1p_far(double x, double u, double m, int e, int key)
{
    asm volatile("");
    const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
    // (1 - (u - x)) when x > 1, else (x - (u - 1))
    const bool big = gt_pos(x, 1.0);
    const double c = (big ? 1.0 : x) - (u - (big ? x : 1.0));
    const double2 t0 = __ldg(reinterpret_cast<const double2*>(f64_log_tab) + 2 * key);       // R, Lh
    const double Ll = __ldg(reinterpret_cast<const double2*>(f64_log_tab) + 2 * key + 1).x;
    const double lg = log1p_series(fma(m, t0.x, -1.0));
    const double ru = f2d_pos(__frcp_rn(f32_rn_pos(u)));   // (double)(1.0f / (float)u)
    const double de = i2d_exact(e);
    return fma(de, ln2_hi, t0.y) + (fma(c, ru, lg) + fma(de, ln2_lo, Ll));
}

__device__ __forceinline__ double series_log1p(double x)
{
    const double u = 1.0 + x;
    const long long ub = bits(u);
    const bool ok = ub > 0LL && ub < 0x7ff0000000000000LL;   // 0 < u < inf
    int e;
    double m = frexp_normal(ok ? u : 1.0, e);   // u >= 2^-53 when ok
    const bool below = bits(m) < bits(0.70710678118654752440);   // m in [1/2, 1/sqrt2): m * 2, exactly
    m = __longlong_as_double(bits(m) + (below ? (1LL << 52) : 0LL));
    e -= below ? 1 : 0;
    const int key = (int)(bits(m) >> 44) - F64_LOG_KEY0;
    const unsigned er = (unsigned)(e - F64_LOG_E0);
    double res;
    if (er < (unsigned)F64_LOG_NE) {
        // (e ln2_hi + Lh, RN(e ln2_lo + Ll)), (R 2^-e, R 2^-e - 1)
        const double2* row = reinterpret_cast<const double2*>(f64_log_e_tab) + 2 * (er * F64_LOG_N + key);
        const double2 hl = __ldg(row), rp = __ldg(row + 1);
        const double lg = log1p_series(fma(x, rp.x, rp.y));
        res = hl.x + (lg + hl.y);
    } else {
        res = log1p_far(x, u, m, e, key);
    }
    const long long special = eq0(u) ? (long long)0xfff0000000000000ULL
                                     : (ub == 0x7ff0000000000000LL ? 0x7ff0000000000000LL
                                                                   : (long long)0xfff8000000000000ULL);
    return __longlong_as_double(ok ? bits(res) : special);   // -inf, +inf, NaN
}

// e^r - 1 by its series to r^5 (the next term is below 1.5e-17 of the
// result); the factor of r^4, 1/24 + r/120, in FP32: scaled by r^4 (below
// 1.7e-10 of the result) its FP32 error stays below 0.1 ulp
__device__ __forceinline__ double expm1_series(double r)
{
    const double r2 = r * r;
    const float pf = __fmaf_rn(0x1.111112p-7f, f32_trunc(r), 0x1.555556p-5f);   // 1/120, 1/24
    double p = fma(f2d_normal(pf), r, 1.0 / 6.0);   // pf near 1/24: normal
    p = fma(p, r, 1.0 / 2.0);
    return fma(r2, p, r);
}

// expm1 for m outside [-2, 1] (rare; out of line, not evaluated
// speculatively): r -= k ln2_lo/256, S = Th em + Tl, (2^m Th - 1) + 2^m S,
// and (Th + S) 2^(m-1023) 2^1023 where 2^m overflows
static __device__ __noinline__ double expm1_far(double r, double dk, int j, int m)
{
    asm volatile("");
    const double ln2_lo = 1.90821492927058770002e-10;
    const double em = expm1_series(fma(dk, -(ln2_lo / 256.0), r));
    const double2 T = __ldg(reinterpret_cast<const double2*>(f64_exp_tab) + j);   // 2^(j/256)
    const double S = fma(T.x, em, T.y);
    if (m > 1023) return ((T.x + S) * pow2i(m - 1023 > 2000 ? 2000 : m - 1023)) * pow2i(1023);
    const double t = pow2i(m < -2000 ? -2000 : m);
    return fma(t, S, fma(t, T.x, -1.0));
}

__device__ __forceinline__ double series_expm1(double w)
{
    const double ln2_hi = 6.93147180369123816490e-01;
    const double wc = __longlong_as_double((abs_lt(w, 800.0) || is_nan(w))
                                               ? bits(w)
                                               : (lt0(w) ? (long long)0xc089000000000000ULL    // -800
                                                         : 0x4089000000000000LL));             // 800
    const float y = __fmul_rn(f32_trunc(wc), 0x1.715476p+8f);   // 256/ln2 in FP32
    const float sh = __fadd_rn(y, 12582912.0f);                  // rounds y to an integer
    const int k = (int)__float_as_uint(sh) - 0x4b400000;
    const int j = k & 255;
    const int m = (k - j) >> 8;
    const double dk = i2d_exact(k);
    // w - k ln2_hi/256, exact (the constant negated, not k: no separate
    // negation of k on the FP64 pipe)
    const double r = fma(dk, -(ln2_hi / 256.0), wc);
    // m in [-2, 1]: e^w - 1 = A em + B, A = e^(k ln2_hi/256) and B = A - 1
    // rounded, from the table, in one fma
    const unsigned mr = (unsigned)(m - F64_EXP_M0);
    if (mr < (unsigned)F64_EXP_NM) {
        const double2 ab = __ldg(reinterpret_cast<const double2*>(f64_exp_ab_tab) + mr * F64_EXP_N + j);
        return fma(ab.x, expm1_series(r), ab.y);
    }
    return expm1_far(r, dk, j, m);
}

// Exit time along one axis from the distance d to the reachable face
// (face = +1, -1, or 0 when no face is reachable: +inf).  Written without
// branches around the quotient and log1p so that the lanes of a warp stay
// converged; lanes with no reachable face compute on harmless operands and
// select +inf.  The values equal those of the branchy form (t1 = d / vp by
// f64_div, z = A t1, t1 when z == 0 else log1p(z) * (1 / A)).
__device__ __forceinline__ double f64_exit_time_d(double A, double iA, double d, double vp, int face)
{
    const double t1 = f64_div(d, face ? vp : 1.0);
    const double z = A * t1;
    const bool lin = eq0(z) || !face;
    const double te = lin ? t1 : series_log1p(lin ? 0.5 : z) * iA;
    return face ? te : CUDART_INF;
}

// the reachable face (v2pos / v1neg: the signs of the face velocities)
__device__ __forceinline__ int f64_face(double vp, bool v2pos, bool v1neg)
{
    return (gt0(vp) && v2pos) ? 1 : ((lt0(vp) && v1neg) ? -1 : 0);
}

// the signed distance to that face (D - pp up, -pp down and otherwise)
__device__ __forceinline__ double f64_face_dist(int face, double D, double pp)
{
    return face > 0 ? D - pp : neg(pp);
}

__device__ __forceinline__ double f64_exit_time(double A, double iA, double D, double vp, double pp, bool v2pos,
                                                bool v1neg, int& face)
{
    face = f64_face(vp, v2pos, v1neg);
    return f64_exit_time_d(A, iA, f64_face_dist(face, D, pp), vp, face);
}

// particle velocity at offset pp from face 1: v1 + A pp, one rounding
__device__ __forceinline__ double f64_vel(double v1, double A, double pp) { return fma(A, pp, v1); }

// analytic motion along one axis for a time dt, clamped to the cell
// (the same values as: vp == 0 or dt == 0 -> pp; w == 0 -> pp + vp dt in one fma;
// else pp + (vp * expm1(w)) * (1 / A), the last product and sum in one
// fma); the operands are selected, so every lane issues one product and
// one fma
__device__ __forceinline__ double f64_move(double A, double iA, double D, double vp, double pp, double dt)
{
    const bool still = eq0(vp) || eq0(dt);
    const double w = A * dt;
    const bool lin = eq0(w);
    const double em = series_expm1(lin ? 0.5 : w);
    const double vem = vp * em;
    double pn = fma(lin ? vp : vem, lin ? dt : iA, pp);
    pn = lt0(pn) ? 0.0 : pn;
    pn = gt_pos(pn, D) ? D : pn;
    return still ? pp : pn;
}

// FP32 estimate of an exit time from an FP32 distance d and the FP64
// particle velocity vp.  Relative error: the truncating conversions and
// the approximate division give ~6e-7 on t1 = d / vp and on z = A t1, and
// d from f32_face_dist below 6.2e-5; g(z) = ln(1 + z) / z is its series
// for |z| < 2^-7, else __logf (absolute error at most 2^-21.41 on [1/2, 2],
// 3 ulp outside) of u = fl(1 + z) over u - 1, in which the rounding of
// 1 + z cancels (Goldberg 1991), or for z < -1/2 of the velocity ratio
// u_exit / vp over z (the ratio, not 1 + z, carries the information
// there): below 4.6e-5, since |ln u| >= 0.0078 wherever __logf is used.  In
// all below 1.2e-4, a quarter of the 2^-11 that the candidate margin of
// 2^-10 allows.  Velocities outside [1e-30, 1e30] (FP32
// could not hold the quotients, and __fdividef gives 0 for divisors
// beyond 2^126) or a NaN mark the estimate as untrusted.
__device__ __forceinline__ float f32_estimate_f(int face, float d, double vp, float fA, float fue, bool& unsafe)
{
    const float vf = f32_trunc(vp);
    const float vs = face ? vf : 1.0f;
    const float t1 = __fdividef(d, vs);
    const float z = fA * t1;
    // both forms, selected (no divergent branch)
    const bool near_m1 = z < -0.5f;
    const float u = 1.0f + z;
    const float L = __logf(near_m1 ? __fdividef(fue, vs) : u);
    const float gl = __fdividef(L, near_m1 ? z : u - 1.0f);
    const float gs = 1.0f + z * (-0.5f + z * (1.0f / 3.0f + z * (-0.25f + z * 0.2f)));
    const float g = fabsf(z) < 0.0078125f ? gs : gl;
    const float e = t1 * g;
    unsafe = face != 0 && (!(fabsf(vf) >= 1e-30f) || !(fabsf(vf) <= 1e30f) || !(e == e));
    return face ? e : CUDART_INF_F;
}

// FP32 distance to the reachable face for the estimates without an FP64
// subtraction: -pp truncated, or D - pp from the truncated operands (error
// below 2^-23 D plus one FP32 rounding, so below 6.2e-5 relative while the
// distance is at least 2^-9 D); nearer the face (rare) the truncated FP64
// difference, out of line
static __device__ __noinline__ float f32_dist_near(double D, double pp) { return f32_trunc(D - pp); }

__device__ __forceinline__ float f32_face_dist(int face, double D, double pp)
{
    const float pf = f32_trunc(pp);
    if (face <= 0) return -pf;
    const float Df = f32_trunc(D);
    const float d = Df - pf;
    return d >= Df * 0x1.0p-9f ? d : f32_dist_near(D, pp);
}

}  // namespace mp
