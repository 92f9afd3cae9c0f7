/*
 * mp_oracle.c - CPU oracle for semi-analytical particle tracking.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path: one particle at a time, one cell at a time, IEEE
 * double precision, no FMA contraction by the compiler (-ffp-contract=off),
 * no vectorisation.
 *
 * What it computes.  The paper (Introduction; Methods, "MODPATH") moves each
 * particle independently with the semi-analytical solution of Pollock (1988):
 * one displacement takes the particle from its position to a face of the
 * current cell, after which it is handed to the neighbour across that face,
 * until a stopping condition holds (a boundary face, the maximum tracking time,
 * a sink cell).  The Pollock solution inside one cell, per axis a:
 *
 *   face velocities   v1 = Q1 / (n * area_a),  v2 = Q2 / (n * area_a)
 *   gradient          A  = (v2 - v1) / D_a            (D_a = cell size)
 *   velocity at p     vp = v1 + A * p                 (p = offset from face 1)
 *   exit time         t_a = ln(v_exit / vp) / A, with d the signed distance
 *                     to the exit face and z = A d / vp (v_exit / vp = 1 + z)
 *   motion            p(t) = p + vp (e^{A t} - 1) / A
 *   and the limits A -> 0: t_a = d / vp, p(t) = p + vp t.
 *
 * Two arithmetic modes evaluate these (opts->arith):
 *
 *   PLAIN, the reference: the formulas as they read, with the A -> 0 limit
 *   built in through the well-conditioned factors log1p(z)/z and
 *   expm1(w)/w:  vp = v1 + A p;  t_a = (d / vp) (log1p(z) / z), z = A (d / vp)
 *   (t_a = d / vp when z == 0);  p(t) = p + (vp t) (expm1(w) / w), w = A t
 *   (p + vp t when w == 0).  log1p and expm1 are the C library's; every
 *   division is IEEE; no fused multiply-add.
 *
 *   MIRROR: the same solution evaluated in Pollock's own forms,
 *   t_a = ln(1 + z) / A and p + vp (e^{A t} - 1) / A, with 1/A formed once
 *   per cell and multiplied, v1 + A p and the motion's last product and sum
 *   as single fused multiply-adds (C99 fma), d / vp as d times a
 *   refined reciprocal (orc_div), and log1p / expm1 evaluated by
 *   fixed table-driven steps (Tang's method: P. T. P. Tang, "Table-driven
 *   implementation of the exponential function in IEEE floating-point
 *   arithmetic", ACM TOMS 15(2), 1989, and "Table-driven implementation of
 *   the logarithm function ...", ACM TOMS 16(4), 1990).  Any other
 *   implementation of these exact steps produces the same bits, which makes
 *   this mode a bit-for-bit check of such an implementation.  Its results
 *   differ from PLAIN's by rounding only (a few ulp per step); the tests
 *   hold both modes to the same pins.
 *
 * A face is reachable on an axis only if the particle velocity and the
 * exit-face velocity point the same way (vp > 0 and v2 > 0 -> face 2;
 * vp < 0 and v1 < 0 -> face 1).  The step time is the smallest reachable t_a
 * (ties go to the lowest axis, x before y before z); the other axes move by
 * the motion formula, the exit axis is set exactly on its face.
 *
 * Readings of points the paper leaves open (it defers the algorithm to
 * Pollock 1988/2016):
 *   - velocities use the cell's own porosity and the cell's own face area;
 *   - z == 0 (and w == 0 in the motion factor) takes the exact limit 1;
 *   - stop at t_stop if t + t_min >= t_stop: every axis moves by t_stop - t;
 *   - no reachable face and t_stop infinite: status NO_EXIT;
 *   - entering an inactive (ibound 0) or constant-head (ibound -1) cell ends
 *     the path (BOUNDARY), entering a sink cell (ibound 2) ends it (SINK,
 *     strong sink), leaving the grid ends it (EXIT_DOMAIN); in all three the
 *     particle stays in its last cell, on the face it left through;
 *   - weak sinks (the paper's default for its second test case: particles
 *     "pass through weak sink cells"): with pass_weak_sinks the particle
 *     enters a sink cell like any other and leaves through a face it can
 *     reach; when no face is reachable inside a sink cell the sink captures
 *     it (SINK) where it is; a particle released in a sink cell stays SINK;
 *     with a weak-sink fraction f > 0 as well, a sink cell whose sink
 *     extracts at least f of its inflow stops particles as a strong sink
 *     does, the others are passed (sink_fraction below);
 *   - a cell-step is one exit-time evaluation, including zero-length steps
 *     and the final partial step; max_steps caps them (STEP_CAP), counted
 *     from the release (a resumed particle carries its count and its hash);
 *   - piecewise-steady flow (Methods, "MODPATH": the outer loop runs over
 *     the flow model's time steps and updates the flow arrays when a step's
 *     end time is reached): each period is one call with t_stop at the
 *     period's end on the period's field, resumed from the previous state;
 *     a moving particle that finds its cell inactive or constant-head under
 *     the new field ends there (BOUNDARY), in a sink cell (SINK) unless weak
 *     sinks are passed;
 *   - pathlines (Methods, "MODPATH": endpoint, timeseries and pathline
 *     simulations): a point at the start and one at the end of every
 *     cell-step (the entry point of the next cell, or where the path ends),
 *     each with its cell, time, step count and status;
 *   - output times t_k are recorded in the step whose interval (t, t + dt]
 *     holds them, with the motion formula at tau = t_k - t on every axis;
 *     t_k at or before the start time records the release position, t_k
 *     after termination records the final position with the final status.
 *
 * Axes: x along column j, y along row i, z along layer k (z grows with k).
 * Offsets p are metres from the cell's low face on each axis.
 */
#include "mp_oracle.h"

#include <math.h>
#include <string.h>

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------- */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t prod = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(prod >> 32);
    *lo = (uint32_t)prod;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in [0, 1) from two 32-bit words */
static double unit53(uint32_t a, uint32_t b)
{
    uint64_t v = (((uint64_t)a << 32) | (uint64_t)b) >> 11;
    return (double)v * (1.0 / 9007199254740992.0);
}

/* ---- grid helpers ------------------------------------------------------ */

static void face_coords(const double* sizes, int n, double origin, double* out /* n+1 */)
{
    out[0] = origin;
    for (int a = 0; a < n; a++) out[a + 1] = out[a] + sizes[a];
}

/* largest index a in [0, n-1] with f[a] <= x (f has n+1 entries); -1 if x
 * lies outside [f[0], f[n]] */
static int locate(const double* f, int n, double x)
{
    if (!(x >= f[0]) || !(x <= f[n])) return -1;
    int a = 0;
    while (a + 1 < n && f[a + 1] <= x) a++;
    return a;
}

static uint64_t fnv_step(uint64_t h, int32_t c)
{
    h ^= (uint64_t)(uint32_t)c;
    h *= 0x100000001b3ULL;
    return h;
}

/* ---- log1p and expm1: argument reduction, a table, a short series ------
 * Both are evaluated with IEEE additions, multiplications and fused
 * multiply-adds (C99 fma, one rounding), exact bit operations on the
 * representation, one FP32 reciprocal and FP32 products, in a fixed order,
 * so that any other implementation of the same steps produces the same
 * bits.  The tables (orc_tables.h, written by gen_tables.py) hold correctly
 * rounded constants.  Accuracy (pinned against the C library in the tests):
 * within a few ulp.
 *
 * log1p(x): u = 1 + x rounded; u = m 2^e with m in [1/sqrt2, sqrt2); the
 * bucket of m (its exponent and top 8 fraction bits) gives R, an 8-bit
 * approximation of 1/m, and -ln R = Lh + Ll.  For e in [-2, 3] (u in
 * [1/(4 sqrt2), 8 sqrt2)): r = (1 + x) R 2^-e - 1 = x R' + (R' - 1) with
 * R' = R 2^-e, in one fma (both terms exact), so r carries the exact
 * 1 + x; otherwise r = m R - 1 (exact: a multiple of 2^-60 below 2^-7, one
 * fma) and the rounding error c of 1 + x (two-sum) enters as c / u, c
 * times the FP32 reciprocal of u.  ln(1 + r) = r - r^2/2 + ... - r^8/8
 * (|r| < 0.006); log1p(x) = (e ln2_hi + Lh) + (ln(1 + r) + (e ln2_lo + Ll))
 * (with c / u added to ln(1 + r) in one fma in the second form), the
 * first sum exact (both terms are multiples of 2^-32).
 * u = +inf gives +inf, u = 0 gives -inf, a NaN gives NaN.
 *
 * expm1(w): |w| limited to 800 (beyond, the result is -1 or +inf either
 * way); k = nearest integer to w 256/ln2, evaluated in FP32 on the
 * significand-truncated w (any nearby integer is a valid reduction);
 * j = k mod 256, m = (k - j)/256; r = w - k ln2_hi/256 (exact);
 * expm1(r) = r + r^2 (1/2 + r/6 + r^2/24 + r^3/120) (|r| < 0.0016).
 * For m in [-2, 1]: expm1(w) = A em + B, A = e^(k ln2_hi/256) and
 * B = A - 1 rounded from the table (the low part of k ln2/256 is in the
 * table).  Otherwise r -= k ln2_lo/256 first; 2^(j/256) = Th + Tl;
 * S = Th expm1(r) + Tl; expm1(w) = (2^m Th - 1) + 2^m S, and for m > 1023
 * (2^m not finite) ((Th + S) 2^(m - 1023)) 2^1023.
 */
#include "orc_tables.h"

static const double ORC_LN2_HI = 6.93147180369123816490e-01;   /* a multiple of 2^-32 */
static const double ORC_LN2_LO = 1.90821492927058770002e-10;

static double orc_from_bits(uint64_t b)
{
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

static uint64_t orc_bits(double v)
{
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    return b;
}

/* FP64 -> FP32 with the significand truncated (magnitudes below the FP32
 * normal range -> signed 0, above it -> signed infinity) */
static float orc_f32_trunc(double x)
{
    uint64_t b = orc_bits(x);
    uint32_t sgn = (uint32_t)(b >> 63) << 31;
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    uint32_t f;
    if (e < -126) f = sgn;
    else if (e > 127) f = sgn | 0x7f800000u;
    else f = sgn | ((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffff);
    float v;
    memcpy(&v, &f, sizeof v);
    return v;
}

/* ln(1 + r) = r + r^2 (-1/2 + r (1/3 + r (-1/4 + r P))), with
 * P = 1/5 - r/6 + r^2/7 - r^3/8 in single precision on the truncated r:
 * it enters scaled by r^5 (|r| < 0.006), below 0.15 ulp of error */
static double orc_log1p_series(double r)
{
    double r2 = r * r;
    float rf = orc_f32_trunc(r);
    float pf = fmaf(-0x1.0p-3f, rf, 0x1.24924ap-3f);     /* -1/8, 1/7 */
    pf = fmaf(pf, rf, -0x1.555556p-3f);                  /* -1/6 */
    pf = fmaf(pf, rf, 0x1.99999ap-3f);                   /* 1/5 */
    double q = fma(r, (double)pf, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    return fma(r2, q, r);
}

double orc_log1p(double x)
{
    double u = 1.0 + x;
    if (!(u > 0.0) || u == INFINITY) return u == 0.0 ? -INFINITY : (u == INFINITY ? INFINITY : NAN);
    int e;
    double m = frexp(u, &e);
    if (m < 0.70710678118654752440) { m = m * 2.0; e = e - 1; }
    int key = (int)(orc_bits(m) >> 44) - ORC_LOG_KEY0;
    double R = orc_from_bits(orc_log_tab[key][0]);
    double Lh = orc_from_bits(orc_log_tab[key][1]);
    double Ll = orc_from_bits(orc_log_tab[key][2]);
    double de = (double)e;
    if (e >= -2 && e <= 3) {
        /* r = (1 + x) R 2^-e - 1 from x itself, to one rounding:
         * x (R 2^-e) + (R 2^-e - 1) in one fma, both terms exact (R has 8
         * significant bits), so the rounding of 1 + x never enters */
        double Rp = ldexp(R, -e);
        double r = fma(x, Rp, Rp - 1.0);
        double lg = orc_log1p_series(r);
        return fma(de, ORC_LN2_HI, Lh) + (lg + fma(de, ORC_LN2_LO, Ll));
    }
    /* other exponents: r = m R - 1 exact, and the rounding error c of
     * 1 + x (two-sum) added as c / u */
    double c = (x > 1.0) ? (1.0 - (u - x)) : (x - (u - 1.0));
    double r = fma(m, R, -1.0);
    double lg = orc_log1p_series(r);
    double ru = (double)(1.0f / (float)u);
    double hi = fma(de, ORC_LN2_HI, Lh);
    double lo = fma(c, ru, lg) + fma(de, ORC_LN2_LO, Ll);
    return hi + lo;
}

/* e^r - 1 = r + r^2 (1/2 + r (1/6 + r P)) to r^5 (|r| < 0.0016: the next
 * term is below 1.5e-17 of the result), with P = 1/24 + r/120 in single
 * precision on the truncated r: scaled by r^4 its error stays below
 * 0.1 ulp */
static double orc_expm1_series(double r)
{
    double r2 = r * r;
    float pf = fmaf(0x1.111112p-7f, orc_f32_trunc(r), 0x1.555556p-5f);   /* 1/120, 1/24 */
    double p = fma((double)pf, r, 1.0 / 6.0);
    p = fma(p, r, 1.0 / 2.0);
    return fma(r2, p, r);
}

double orc_expm1(double w)
{
    double wc = w;
    if (fabs(w) > 800.0) wc = w < 0.0 ? -800.0 : 800.0;
    float y = orc_f32_trunc(wc) * 0x1.715476p+8f;          /* 256/ln2 rounded to FP32 */
    float sh = y + 12582912.0f;                            /* 1.5 2^23: rounds y to an integer */
    uint32_t sb;
    memcpy(&sb, &sh, sizeof sb);
    int k = (int)sb - 0x4b400000;
    int j = k & 255;
    int m = (k - j) / 256;
    double dk = (double)k;
    double r = fma(-dk, ORC_LN2_HI / 256.0, wc);           /* exact */
    if (m >= ORC_EXP_M0 && m < ORC_EXP_M0 + ORC_EXP_NM) {
        /* e^w - 1 = e^(k ln2_hi/256) (1 + em) - 1 = A em + B with
         * em = e^r - 1, A = e^(k ln2_hi/256) and B = A - 1 rounded from
         * the table: one fma */
        double A = orc_from_bits(orc_exp_ab[m - ORC_EXP_M0][j][0]);
        double B = orc_from_bits(orc_exp_ab[m - ORC_EXP_M0][j][1]);
        return fma(A, orc_expm1_series(r), B);
    }
    r = fma(-dk, ORC_LN2_LO / 256.0, r);
    double em = orc_expm1_series(r);
    double Th = orc_from_bits(orc_exp_tab[j][0]);
    double Tl = orc_from_bits(orc_exp_tab[j][1]);
    double S = fma(Th, em, Tl);
    if (m > 1023) return ((Th + S) * ldexp(1.0, m - 1023)) * ldexp(1.0, 1023);
    double t = ldexp(1.0, m);
    return fma(t, S, fma(t, Th, -1.0));
}

/* d / v as d times a reciprocal: the IEEE single-precision reciprocal y0
 * of the truncated v, then one third-order step y = y0 + y0 (e + e^2) with
 * e = 1 - v y0 in one fma (rounded by less than 2^-75): the truncated
 * series of 1/v = y0 / (1 - e) leaves e^3 < 2^-67 and the
 * roundings (1 / v within about half an ulp, the quotient within about
 * one); |v| outside [2^-120, 2^121), 0, infinity and NaN divide in IEEE
 * double */
double orc_div(double d, double v)
{
    int e = (int)((orc_bits(v) >> 52) & 0x7ff) - 1023;
    if (e < -120 || e > 120) return d / v;
    double y = (double)(1.0f / orc_f32_trunc(v));
    double e0 = fma(-v, y, 1.0);
    y = fma(y, fma(e0, e0, e0), y);
    return d * y;
}

/* ---- the Pollock pieces ---------------------------------------------- */

double orc_exit_time(double v1, double v2, double A, double iA, double D, double p, int* face)
{
    double vp = fma(A, p, v1);
    double d;
    if (vp > 0.0 && v2 > 0.0) { *face = 1; d = D - p; }
    else if (vp < 0.0 && v1 < 0.0) { *face = -1; d = -p; }
    else { *face = 0; return INFINITY; }
    double t1 = orc_div(d, vp);
    double z = A * t1;
    if (z == 0.0) return t1;
    return orc_log1p(z) * iA;
}

double orc_move(double v1, double A, double iA, double D, double p, double dt)
{
    double vp = fma(A, p, v1);
    /* no motion when vp or dt is zero (the plain mode tests the product,
     * which differs only where vp dt underflows) */
    if (vp == 0.0 || dt == 0.0) return p;
    double w = A * dt;
    double pn = (w == 0.0) ? fma(vp, dt, p) : fma(vp * orc_expm1(w), iA, p);
    if (pn < 0.0) pn = 0.0;
    if (pn > D) pn = D;
    return pn;
}

/* ---- the plain reading (PLAIN mode) -------------------------------- */

double orc_exit_time_plain(double v1, double v2, double A, double D, double p, int* face)
{
    double vp = v1 + A * p;
    double d;
    if (vp > 0.0 && v2 > 0.0) { *face = 1; d = D - p; }
    else if (vp < 0.0 && v1 < 0.0) { *face = -1; d = -p; }
    else { *face = 0; return INFINITY; }
    double t1 = d / vp;
    double z = A * t1;
    if (z == 0.0) return t1;
    return t1 * (log1p(z) / z);
}

double orc_move_plain(double v1, double A, double D, double p, double dt)
{
    double vp = v1 + A * p;
    double s = vp * dt;
    if (s == 0.0) return p;
    double w = A * dt;
    double pn = (w == 0.0) ? p + s : p + s * (expm1(w) / w);
    if (pn < 0.0) pn = 0.0;
    if (pn > D) pn = D;
    return pn;
}

/* ---- cell data gathered at cell entry (the per-cell "initialisation") -- */

typedef struct {
    double v1[3], v2[3], A[3], iA[3], D[3];
} cellvel;

static void cell_velocities(const orc_field* f, int k, int i, int j, cellvel* cv)
{
    const int nrow = f->nrow, ncol = f->ncol, nlay = f->nlay;
    size_t c = ((size_t)k * nrow + i) * ncol + j;
    double n = f->porosity[c];
    double dx = f->delr[j], dy = f->delc[i], dzz = f->dz[k];
    double ax = dy * dzz, ay = dx * dzz, az = dx * dy;
    double qx1 = f->qx[((size_t)k * nrow + i) * (ncol + 1) + j];
    double qx2 = f->qx[((size_t)k * nrow + i) * (ncol + 1) + j + 1];
    double qy1 = f->qy[((size_t)k * (nrow + 1) + i) * ncol + j];
    double qy2 = f->qy[((size_t)k * (nrow + 1) + i + 1) * ncol + j];
    double qz1 = f->qz[((size_t)k * nrow + i) * ncol + j];
    double qz2 = f->qz[((size_t)(k + 1) * nrow + i) * ncol + j];
    (void)nlay;
    cv->v1[0] = qx1 / (n * ax); cv->v2[0] = qx2 / (n * ax);
    cv->v1[1] = qy1 / (n * ay); cv->v2[1] = qy2 / (n * ay);
    cv->v1[2] = qz1 / (n * az); cv->v2[2] = qz2 / (n * az);
    cv->D[0] = dx; cv->D[1] = dy; cv->D[2] = dzz;
    for (int a = 0; a < 3; a++) {
        cv->A[a] = (cv->v2[a] - cv->v1[a]) / cv->D[a];
        cv->iA[a] = (cv->A[a] != 0.0) ? 1.0 / cv->A[a] : 0.0;
    }
}

/* the exit time and the motion of axis a in the mode opt->arith selects */
static double ex_time(const orc_track_opts* opt, const cellvel* cv, int a, double p, int* face)
{
    if (opt->arith == ORC_ARITH_MIRROR)
        return orc_exit_time(cv->v1[a], cv->v2[a], cv->A[a], cv->iA[a], cv->D[a], p, face);
    return orc_exit_time_plain(cv->v1[a], cv->v2[a], cv->A[a], cv->D[a], p, face);
}

static double mv(const orc_track_opts* opt, const cellvel* cv, int a, double p, double dt)
{
    if (opt->arith == ORC_ARITH_MIRROR)
        return orc_move(cv->v1[a], cv->A[a], cv->iA[a], cv->D[a], p, dt);
    return orc_move_plain(cv->v1[a], cv->A[a], cv->D[a], p, dt);
}

/* ---- release ----------------------------------------------------------- */

int orc_release_box(const orc_field* f, int64_t n, const double lo[3], const double hi[3],
                    uint64_t seed, uint64_t id_offset,
                    int32_t* cell, double* px, double* py, double* pz, uint8_t* status)
{
    const int nlay = f->nlay, nrow = f->nrow, ncol = f->ncol;
    double xf[ORC_MAX_AXIS + 1], yf[ORC_MAX_AXIS + 1], zf[ORC_MAX_AXIS + 1];
    if (ncol > ORC_MAX_AXIS || nrow > ORC_MAX_AXIS || nlay > ORC_MAX_AXIS) return -1;
    face_coords(f->delr, ncol, f->origin[0], xf);
    face_coords(f->delc, nrow, f->origin[1], yf);
    face_coords(f->dz, nlay, f->origin[2], zf);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t q = 0; q < n; q++) {
        uint64_t id = (uint64_t)q + id_offset;
        uint32_t c0[4] = {(uint32_t)id, (uint32_t)(id >> 32), 0u, 0u};
        uint32_t c1[4] = {(uint32_t)id, (uint32_t)(id >> 32), 1u, 0u};
        uint32_t r[4], s[4];
        orc_philox4x32_10(c0, key, r);
        orc_philox4x32_10(c1, key, s);
        double ux = unit53(r[0], r[1]), uy = unit53(r[2], r[3]), uz = unit53(s[0], s[1]);
        double gx = lo[0] + ux * (hi[0] - lo[0]);
        double gy = lo[1] + uy * (hi[1] - lo[1]);
        double gz = lo[2] + uz * (hi[2] - lo[2]);
        int j = locate(xf, ncol, gx), i = locate(yf, nrow, gy), k = locate(zf, nlay, gz);
        if (j < 0 || i < 0 || k < 0) {
            cell[q] = -1; px[q] = 0.0; py[q] = 0.0; pz[q] = 0.0;
            status[q] = ORC_ST_INVALID_RELEASE;
            continue;
        }
        double ox = gx - xf[j], oy = gy - yf[i], oz = gz - zf[k];
        if (ox < 0.0) ox = 0.0;
        if (ox > f->delr[j]) ox = f->delr[j];
        if (oy < 0.0) oy = 0.0;
        if (oy > f->delc[i]) oy = f->delc[i];
        if (oz < 0.0) oz = 0.0;
        if (oz > f->dz[k]) oz = f->dz[k];
        int32_t c = (int32_t)(((int64_t)k * nrow + i) * ncol + j);
        cell[q] = c; px[q] = ox; py[q] = oy; pz[q] = oz;
        int8_t ib = f->ibound[c];
        status[q] = (ib == 1) ? ORC_ST_ACTIVE : (ib == 2) ? ORC_ST_SINK : ORC_ST_INVALID_RELEASE;
    }
    return 0;
}

int orc_release_explicit(const orc_field* f, int64_t n, const int32_t* cell_in, const double* frac,
                         int32_t* cell, double* px, double* py, double* pz, uint8_t* status)
{
    const int nlay = f->nlay, nrow = f->nrow, ncol = f->ncol;
    const int64_t ncell = (int64_t)nlay * nrow * ncol;
    for (int64_t q = 0; q < n; q++) {
        int32_t c = cell_in[q];
        if (c < 0 || c >= ncell) {
            cell[q] = -1; px[q] = py[q] = pz[q] = 0.0; status[q] = ORC_ST_INVALID_RELEASE;
            continue;
        }
        int j = c % ncol, i = (c / ncol) % nrow, k = c / (ncol * nrow);
        double fx = frac[3 * q], fy = frac[3 * q + 1], fz = frac[3 * q + 2];
        if (fx < 0.0) fx = 0.0;
        if (fx > 1.0) fx = 1.0;
        if (fy < 0.0) fy = 0.0;
        if (fy > 1.0) fy = 1.0;
        if (fz < 0.0) fz = 0.0;
        if (fz > 1.0) fz = 1.0;
        cell[q] = c;
        px[q] = fx * f->delr[j]; py[q] = fy * f->delc[i]; pz[q] = fz * f->dz[k];
        int8_t ib = f->ibound[c];
        status[q] = (ib == 1) ? ORC_ST_ACTIVE : (ib == 2) ? ORC_ST_SINK : ORC_ST_INVALID_RELEASE;
    }
    return 0;
}

/* ---- jitter (test instrument) ------------------------------------------- */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) finaliser of a counter */
static uint64_t splitmix64(uint64_t x)
{
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

/* uniform in [-1, 1) for (seed, particle, step, slot) */
static double jitter_u(uint64_t seed, int64_t q, int64_t step, int slot)
{
    uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)q ^ splitmix64(((uint64_t)step << 3) | (uint64_t)slot)));
    return (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* ---- tracking ------------------------------------------------------------ */

static void write_record(const orc_track_out* o, int64_t n, int kk, int64_t q,
                         double gx, double gy, double gz, int32_t cell, uint8_t st)
{
    size_t r = (size_t)kk * (size_t)n + (size_t)q;
    o->ts_x[r] = gx; o->ts_y[r] = gy; o->ts_z[r] = gz;
    o->ts_cell[r] = cell; o->ts_status[r] = st;
}

static void path_point(const orc_track_out* o, int64_t q, double x, double y, double z, double t,
                       int32_t cell, int64_t seq, uint8_t st)
{
    if (!o->path) return;
    int64_t r = (*o->path_n)++;
    if (r >= o->path_cap) return;
    orc_path_rec* e = &o->path[r];
    e->x = x; e->y = y; e->z = z; e->t = t;
    e->particle = (int32_t)q; e->cell = cell; e->seq = (uint32_t)seq; e->status = st;
    e->pad[0] = e->pad[1] = e->pad[2] = 0;
}

static void trace_step(const orc_track_out* o, int64_t q, int32_t cell, double t, const cellvel* cv,
                       const orc_track_opts* opt, const double p[3], const double te[3], const int face[3],
                       int ax)
{
    int64_t r = (*o->trace_n)++;
    if (r >= o->trace_cap) return;
    orc_trace_rec* e = &o->trace[r];
    memset(e, 0, sizeof *e);
    for (int a = 0; a < 3; a++) {
        e->te[a] = te[a];
        e->vp[a] = (opt->arith == ORC_ARITH_MIRROR) ? fma(cv->A[a], p[a], cv->v1[a]) : cv->v1[a] + cv->A[a] * p[a];
        e->vf[a] = fmax(fabs(cv->v1[a]), fabs(cv->v2[a]));
        e->face[a] = (int8_t)face[a];
    }
    e->t = t;
    e->particle = (int32_t)q;
    e->cell = cell;
    e->ax = (int8_t)ax;
}

/* ---- grids ---------------------------------------------------------------
 * The tracking loop sees a grid through three questions: the box of a cell
 * (low corner, sizes), the cell's Pollock velocities, and the cell across a
 * face at a given exit point (-1 outside the domain). */

struct orc_grid {
    void (*box)(const orc_grid* g, int32_t c, double o[3], double D[3]);
    void (*vel)(const orc_grid* g, int32_t c, cellvel* cv);
    void (*flows)(const orc_grid* g, int32_t c, double q[6]);   /* total flow per face, +axis direction */
    int32_t (*across)(const orc_grid* g, int32_t c, int ax, int side, double x[3]);
    const int8_t* ibound;
    const orc_field* f;
    const orc_usg_field* u;
    const double *xf, *yf, *zf;
};

static void st_box(const orc_grid* g, int32_t c, double o[3], double D[3])
{
    const orc_field* f = g->f;
    int j = c % f->ncol, i = (c / f->ncol) % f->nrow, k = c / (f->ncol * f->nrow);
    o[0] = g->xf[j]; o[1] = g->yf[i]; o[2] = g->zf[k];
    D[0] = f->delr[j]; D[1] = f->delc[i]; D[2] = f->dz[k];
}

static void st_vel(const orc_grid* g, int32_t c, cellvel* cv)
{
    const orc_field* f = g->f;
    cell_velocities(f, c / (f->ncol * f->nrow), (c / f->ncol) % f->nrow, c % f->ncol, cv);
}

static void st_flows(const orc_grid* g, int32_t c, double q[6])
{
    const orc_field* f = g->f;
    const int nrow = f->nrow, ncol = f->ncol;
    int j = c % ncol, i = (c / ncol) % nrow, k = c / (ncol * nrow);
    q[0] = f->qx[((size_t)k * nrow + i) * (ncol + 1) + j];
    q[1] = f->qx[((size_t)k * nrow + i) * (ncol + 1) + j + 1];
    q[2] = f->qy[((size_t)k * (nrow + 1) + i) * ncol + j];
    q[3] = f->qy[((size_t)k * (nrow + 1) + i + 1) * ncol + j];
    q[4] = f->qz[((size_t)k * nrow + i) * ncol + j];
    q[5] = f->qz[((size_t)(k + 1) * nrow + i) * ncol + j];
}

static int32_t st_across(const orc_grid* g, int32_t c, int ax, int side, double x[3])
{
    const orc_field* f = g->f;
    (void)x;
    int j = c % f->ncol, i = (c / f->ncol) % f->nrow, k = c / (f->ncol * f->nrow);
    if (ax == 0) j += side;
    else if (ax == 1) i += side;
    else k += side;
    if (j < 0 || j >= f->ncol || i < 0 || i >= f->nrow || k < 0 || k >= f->nlay) return -1;
    return (int32_t)(((int64_t)k * f->nrow + i) * f->ncol + j);
}

/* rectangular unstructured cells: face velocities from the total flow of
 * each face (its sub-faces summed in list order), the cell's own face area */
static void usg_box(const orc_grid* g, int32_t c, double o[3], double D[3])
{
    const double* b = g->u->box + 6 * (size_t)c;
    o[0] = b[0]; o[1] = b[1]; o[2] = b[2];
    D[0] = b[3]; D[1] = b[4]; D[2] = b[5];
}

static double usg_face_flow(const orc_usg_field* u, int32_t c, int fi)
{
    const int64_t e0 = u->face_off[6 * (size_t)c + fi], e1 = u->face_off[6 * (size_t)c + fi + 1];
    if (e1 <= e0) return 0.0;
    double s = u->q[e0];
    for (int64_t e = e0 + 1; e < e1; e++) s += u->q[e];
    return s;
}

static void usg_flows(const orc_grid* g, int32_t c, double q[6])
{
    for (int fi = 0; fi < 6; fi++) q[fi] = usg_face_flow(g->u, c, fi);
}

static void usg_vel(const orc_grid* g, int32_t c, cellvel* cv)
{
    const orc_usg_field* u = g->u;
    const double* b = u->box + 6 * (size_t)c;
    double n = u->porosity[c];
    double dx = b[3], dy = b[4], dzz = b[5];
    double ax = dy * dzz, ay = dx * dzz, az = dx * dy;
    cv->v1[0] = usg_face_flow(u, c, 0) / (n * ax); cv->v2[0] = usg_face_flow(u, c, 1) / (n * ax);
    cv->v1[1] = usg_face_flow(u, c, 2) / (n * ay); cv->v2[1] = usg_face_flow(u, c, 3) / (n * ay);
    cv->v1[2] = usg_face_flow(u, c, 4) / (n * az); cv->v2[2] = usg_face_flow(u, c, 5) / (n * az);
    cv->D[0] = dx; cv->D[1] = dy; cv->D[2] = dzz;
    for (int a = 0; a < 3; a++) {
        cv->A[a] = (cv->v2[a] - cv->v1[a]) / cv->D[a];
        cv->iA[a] = (cv->A[a] != 0.0) ? 1.0 / cv->A[a] : 0.0;
    }
}

/* The neighbour across face (ax, side) at the exit point x: the sub-face
 * whose rectangle holds x (first in list order; else the nearest, by the
 * larger of the two axis distances, first on ties), provided its flow runs
 * in the crossing direction; otherwise the nearest sub-face whose flow does
 * (one exists: the face's total flow has that sign, or the particle would
 * not have left through it), and x moves onto that sub-face's rectangle.
 * No sub-face: outside. */
static double rect_dist(const double* r, double xa, double xb)
{
    double da = fmax(r[0] - xa, xa - r[1]);
    double db = fmax(r[2] - xb, xb - r[3]);
    return fmax(fmax(da, db), 0.0);
}

static int32_t usg_across(const orc_grid* g, int32_t c, int ax, int side, double x[3])
{
    const orc_usg_field* u = g->u;
    const int fi = 2 * ax + (side > 0 ? 1 : 0);
    const int64_t e0 = u->face_off[6 * (size_t)c + fi], e1 = u->face_off[6 * (size_t)c + fi + 1];
    if (e1 <= e0) return -1;
    const int oa = ax == 0 ? 1 : 0, ob = ax == 2 ? 1 : 2;
    const double xa = x[oa], xb = x[ob];
    int64_t best = e0;
    double bd = INFINITY;
    for (int64_t e = e0; e < e1; e++) {
        const double d = rect_dist(u->rect + 4 * (size_t)e, xa, xb);
        if (d < bd) { bd = d; best = e; }
        if (d == 0.0) break;
    }
    if (u->q[best] * (double)side > 0.0) return u->nbr[best];
    int64_t alt = -1;
    double ad = INFINITY;
    for (int64_t e = e0; e < e1; e++) {
        if (!(u->q[e] * (double)side > 0.0)) continue;
        const double d = rect_dist(u->rect + 4 * (size_t)e, xa, xb);
        if (d < ad) { ad = d; alt = e; }
    }
    if (alt < 0) return u->nbr[best];
    const double* r = u->rect + 4 * (size_t)alt;
    x[oa] = fmin(fmax(xa, r[0]), r[1]);
    x[ob] = fmin(fmax(xb, r[2]), r[3]);
    return u->nbr[alt];
}

/* Weak sinks with a threshold (Introduction: how weak sink cells are
 * treated is a choice of the tracking configuration): the fraction of a
 * cell's inflow its sink extracts, from the volume balance of its face
 * flows (inflow: flow entering through a face; extraction: inflow minus
 * outflow), summed face by face in the order x1, x2, y1, y2, z1, z2; a cell
 * without inflow counts as extracting all of it. */
static double sink_fraction(const orc_grid* g, int32_t c)
{
    double q[6];
    g->flows(g, c, q);
    double in = 0.0, out = 0.0;
    for (int a = 0; a < 3; a++) {
        const double q1 = q[2 * a], q2 = q[2 * a + 1];
        if (q1 > 0.0) in += q1; else out += -q1;   /* low face: +axis flow enters */
        if (q2 < 0.0) in += -q2; else out += q2;   /* high face: +axis flow leaves */
    }
    return in > 0.0 ? (in - out) / in : 1.0;
}

/* a sink cell stops particles (entering it or released in it): always
 * without pass-through; with it, when its sink extracts at least
 * weak_sink_fraction (> 0) of its inflow */
static int sink_stops(const orc_grid* g, int32_t c, const orc_track_opts* opt)
{
    if (!opt->pass_weak_sinks) return 1;
    return opt->weak_sink_fraction > 0.0 && sink_fraction(g, c) >= opt->weak_sink_fraction;
}

static int track_core(const orc_grid* g, int64_t n,
                      const int32_t* cell0, const double* px0, const double* py0, const double* pz0,
                      const double* t0, const uint8_t* status0, const uint32_t* steps0, const uint64_t* hash0,
                      const uint8_t* face0, const orc_track_opts* opt, const orc_track_out* out)
{
    const double t_stop = opt->t_stop;
    const int nt = (opt->times && out->ts_x) ? opt->n_times : 0;
    const int64_t max_steps = opt->max_steps > 0 ? opt->max_steps : ORC_DEFAULT_MAX_STEPS;

    for (int64_t q = 0; q < n; q++) {
        int32_t c = cell0[q];
        uint8_t st = status0 ? status0[q] : ORC_ST_ACTIVE;
        double p[3] = {px0[q], py0[q], pz0[q]};
        double t = t0 ? t0[q] : 0.0;
        int64_t steps = steps0 ? (int64_t)steps0[q] : 0;
        uint8_t exit_face = (steps > 0 && face0) ? face0[q] : ORC_FACE_NONE;
        uint64_t h = 0xcbf29ce484222325ULL;
        int kn = 0;
        double o[3] = {0.0, 0.0, 0.0}, D[3] = {0.0, 0.0, 0.0};   /* the cell's low corner and sizes */
        if (c >= 0) {
            g->box(g, c, o, D);
            h = (steps > 0 && hash0) ? hash0[q] : fnv_step(h, c);
            /* a moving particle in a cell that is not active under this
             * field (a later flow period can change ibound) stops there */
            if (st == ORC_ST_ACTIVE) {
                int8_t ib0 = g->ibound[c];
                if (ib0 == 0 || ib0 == -1) st = ORC_ST_BOUNDARY;
                else if (ib0 == 2 && sink_stops(g, c, opt)) st = ORC_ST_SINK;
            }
        } else {
            st = ORC_ST_INVALID_RELEASE;
        }
        /* jitter (test instrument): the start position, as it would be
         * rounded when a reduced-precision evaluation loads it */
        if (opt->jitter > 0.0 && c >= 0 && st == ORC_ST_ACTIVE) {
            for (int a = 0; a < 3; a++) {
                double pa = p[a] + opt->jitter * jitter_u(opt->jitter_seed, opt->jitter_id0 + q, steps, 4 + a) * D[a];
                p[a] = pa < 0.0 ? 0.0 : (pa > D[a] ? D[a] : pa);
            }
        }
        /* output times at or before the start: the release position */
        while (kn < nt && opt->times[kn] <= t) {
            if (c >= 0)
                write_record(out, n, kn, q, o[0] + p[0], o[1] + p[1], o[2] + p[2], c, st);
            else
                write_record(out, n, kn, q, NAN, NAN, NAN, -1, st);
            kn++;
        }
        /* pathline: the start point, with the status it starts with */
        if (opt->path_start && c >= 0)
            path_point(out, q, o[0] + p[0], o[1] + p[1], o[2] + p[2], t, c, steps, st);
        int took = 0;   /* the last loop pass took a cell-step */
        while (st == ORC_ST_ACTIVE) {
            took = 0;
            if (t >= t_stop) { st = ORC_ST_TIME; break; }
            if (steps >= max_steps) { st = ORC_ST_STEP_CAP; break; }
            cellvel cv;
            g->vel(g, c, &cv);
            int face[3];
            double te[3];
            for (int a = 0; a < 3; a++)
                te[a] = ex_time(opt, &cv, a, p[a], &face[a]);
            int ax = -1;
            double tmin = INFINITY;
            for (int a = 0; a < 3; a++)
                if (face[a] != 0 && te[a] < tmin) { tmin = te[a]; ax = a; }
            steps++;
            took = 1;
            if (out->trace) trace_step(out, q, c, t, &cv, opt, p, te, face,
                                       (ax >= 0 && t + tmin < t_stop) ? ax : -1);
            if (ax < 0 && g->ibound[c] == 2) {
                /* inside a sink cell with no reachable face: captured */
                st = ORC_ST_SINK;
                break;
            }
            if (ax < 0 && !(t_stop < INFINITY)) {
                /* no reachable face and no stop time: the particle stays in
                 * this cell; later output times still see it move inside */
                while (kn < nt) {
                    double tau = opt->times[kn] - t;
                    double g0 = o[0] + mv(opt, &cv, 0, p[0], tau);
                    double g1 = o[1] + mv(opt, &cv, 1, p[1], tau);
                    double g2 = o[2] + mv(opt, &cv, 2, p[2], tau);
                    write_record(out, n, kn, q, g0, g1, g2, c, ORC_ST_NO_EXIT);
                    kn++;
                }
                st = ORC_ST_NO_EXIT;
                break;
            }
            if (ax < 0 || t + tmin >= t_stop) {
                double dt = t_stop - t;
                while (kn < nt && opt->times[kn] <= t_stop) {
                    double tau = opt->times[kn] - t;
                    double g0 = o[0] + mv(opt, &cv, 0, p[0], tau);
                    double g1 = o[1] + mv(opt, &cv, 1, p[1], tau);
                    double g2 = o[2] + mv(opt, &cv, 2, p[2], tau);
                    write_record(out, n, kn, q, g0, g1, g2, c, ORC_ST_ACTIVE);
                    kn++;
                }
                for (int a = 0; a < 3; a++) p[a] = mv(opt, &cv, a, p[a], dt);
                t = t_stop;
                st = ORC_ST_TIME;
                break;
            }
            /* displacement to the exit face of axis ax */
            double dt = tmin;
            if (opt->jitter > 0.0) dt = dt * (1.0 + opt->jitter * jitter_u(opt->jitter_seed, opt->jitter_id0 + q, steps, 0));
            double t_end = t + dt;
            while (kn < nt && opt->times[kn] <= t_end) {
                double tau = opt->times[kn] - t;
                double g0 = o[0] + mv(opt, &cv, 0, p[0], tau);
                double g1 = o[1] + mv(opt, &cv, 1, p[1], tau);
                double g2 = o[2] + mv(opt, &cv, 2, p[2], tau);
                write_record(out, n, kn, q, g0, g1, g2, c, ORC_ST_ACTIVE);
                kn++;
            }
            for (int a = 0; a < 3; a++) {
                if (a == ax) p[a] = (face[a] > 0) ? cv.D[a] : 0.0;
                else p[a] = mv(opt, &cv, a, p[a], dt);
            }
            t = t_end;
            exit_face = (uint8_t)(2 * ax + (face[ax] > 0 ? 1 : 0));
            /* hand over to the neighbour across the exit face (at the exit point) */
            const int side = face[ax];
            double xg[3] = {o[0] + p[0], o[1] + p[1], o[2] + p[2]};
            const int32_t nc = g->across(g, c, ax, side, xg);
            if (nc < 0) {
                st = ORC_ST_EXIT_DOMAIN;
                break;
            }
            int8_t ib = g->ibound[nc];
            if (ib == 0 || ib == -1) { st = ORC_ST_BOUNDARY; break; }
            if (ib == 2 && sink_stops(g, nc, opt)) { st = ORC_ST_SINK; break; }
            double on[3], Dn[3];
            g->box(g, nc, on, Dn);
            /* the other axes keep their global coordinate (o - on is 0
             * between cells of one column of a rectilinear grid), clamped
             * to the new cell; the exit axis enters on the shared face */
            for (int a = 0; a < 3; a++) {
                if (a == ax) continue;
                /* a hand-over that moved the point along the face (see
                 * usg_across) enters at the moved point */
                double pa = (xg[a] == o[a] + p[a]) ? p[a] + (o[a] - on[a]) : xg[a] - on[a];
                if (pa < 0.0) pa = 0.0;
                if (pa > Dn[a]) pa = Dn[a];
                p[a] = pa;
            }
            p[ax] = (side > 0) ? 0.0 : Dn[ax];
            if (opt->jitter > 0.0) {
                for (int a = 0; a < 3; a++) {
                    if (a == ax) continue;
                    double pa = p[a] + opt->jitter * jitter_u(opt->jitter_seed, opt->jitter_id0 + q, steps, 1 + a) * Dn[a];
                    p[a] = pa < 0.0 ? 0.0 : (pa > Dn[a] ? Dn[a] : pa);
                }
            }
            c = nc;
            for (int a = 0; a < 3; a++) { o[a] = on[a]; D[a] = Dn[a]; }
            h = fnv_step(h, c);
            /* pathline: the entry point in the new cell */
            path_point(out, q, o[0] + p[0], o[1] + p[1], o[2] + p[2], t, c, steps, ORC_ST_ACTIVE);
        }
        /* pathline: where the last step ended (stop time, sink, boundary, ...) */
        if (took) path_point(out, q, o[0] + p[0], o[1] + p[1], o[2] + p[2], t, c, steps, st);
        /* output times after termination: the final position */
        while (kn < nt) {
            if (c >= 0)
                write_record(out, n, kn, q, o[0] + p[0], o[1] + p[1], o[2] + p[2], c, st);
            else
                write_record(out, n, kn, q, NAN, NAN, NAN, -1, st);
            kn++;
        }
        if (out->cell) out->cell[q] = c;
        if (out->px) {
            out->px[q] = p[0]; out->py[q] = p[1]; out->pz[q] = p[2];
        }
        if (out->gx) {
            if (c >= 0) {
                out->gx[q] = o[0] + p[0]; out->gy[q] = o[1] + p[1]; out->gz[q] = o[2] + p[2];
            } else {
                out->gx[q] = NAN; out->gy[q] = NAN; out->gz[q] = NAN;
            }
        }
        if (out->t) out->t[q] = t;
        if (out->status) out->status[q] = st;
        if (out->steps) out->steps[q] = (uint32_t)steps;
        if (out->exit_face) out->exit_face[q] = exit_face;
        if (out->hash) out->hash[q] = h;
    }
    return 0;
}

int orc_track(const orc_field* f, int64_t n,
              const int32_t* cell0, const double* px0, const double* py0, const double* pz0,
              const double* t0, const uint8_t* status0, const uint32_t* steps0, const uint64_t* hash0,
              const uint8_t* face0, const orc_track_opts* opt, const orc_track_out* out)
{
    double xf[ORC_MAX_AXIS + 1], yf[ORC_MAX_AXIS + 1], zf[ORC_MAX_AXIS + 1];
    if (f->ncol > ORC_MAX_AXIS || f->nrow > ORC_MAX_AXIS || f->nlay > ORC_MAX_AXIS) return -1;
    face_coords(f->delr, f->ncol, f->origin[0], xf);
    face_coords(f->delc, f->nrow, f->origin[1], yf);
    face_coords(f->dz, f->nlay, f->origin[2], zf);
    orc_grid g = {st_box, st_vel, st_flows, st_across, f->ibound, f, NULL, xf, yf, zf};
    return track_core(&g, n, cell0, px0, py0, pz0, t0, status0, steps0, hash0, face0, opt, out);
}

int orc_usg_track(const orc_usg_field* u, int64_t n,
                  const int32_t* cell0, const double* px0, const double* py0, const double* pz0,
                  const double* t0, const uint8_t* status0, const uint32_t* steps0, const uint64_t* hash0,
                  const uint8_t* face0, const orc_track_opts* opt, const orc_track_out* out)
{
    orc_grid g = {usg_box, usg_vel, usg_flows, usg_across, u->ibound, NULL, u, NULL, NULL, NULL};
    return track_core(&g, n, cell0, px0, py0, pz0, t0, status0, steps0, hash0, face0, opt, out);
}

int orc_usg_release_explicit(const orc_usg_field* u, int64_t n, const int32_t* cell_in, const double* frac,
                             int32_t* cell, double* px, double* py, double* pz, uint8_t* status)
{
    for (int64_t q = 0; q < n; q++) {
        int32_t c = cell_in[q];
        if (c < 0 || c >= u->ncell) {
            cell[q] = -1; px[q] = py[q] = pz[q] = 0.0; status[q] = ORC_ST_INVALID_RELEASE;
            continue;
        }
        const double* b = u->box + 6 * (size_t)c;
        double fx = frac[3 * q], fy = frac[3 * q + 1], fz = frac[3 * q + 2];
        if (fx < 0.0) fx = 0.0;
        if (fx > 1.0) fx = 1.0;
        if (fy < 0.0) fy = 0.0;
        if (fy > 1.0) fy = 1.0;
        if (fz < 0.0) fz = 0.0;
        if (fz > 1.0) fz = 1.0;
        cell[q] = c;
        px[q] = fx * b[3]; py[q] = fy * b[4]; pz[q] = fz * b[5];
        int8_t ib = u->ibound[c];
        status[q] = (ib == 1) ? ORC_ST_ACTIVE : (ib == 2) ? ORC_ST_SINK : ORC_ST_INVALID_RELEASE;
    }
    return 0;
}
