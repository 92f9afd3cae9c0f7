/*
 * fieldgen.c - steady finite-volume head solve for synthetic MODFLOW-style
 * flow fields (input generation only; none of the particle-tracking
 * arithmetic lives here).
 *
 * Grid: nlay x nrow x ncol cells, linear index c = (k*nrow + i)*ncol + j,
 * rectilinear spacing delr[ncol] (x, along j), delc[nrow] (y, along i),
 * dz[nlay] (z, along k).  ibound: 0 inactive, 1 active, -1 constant head,
 * 2 active cell that is a strong sink for tracking (a well; for the head
 * solve it is an ordinary unknown with a source term).
 *
 * The 7-point finite-volume system uses harmonic-mean inter-cell
 * conductances C = 2 A / (d_a/K_a + d_b/K_b).  Every active cell balances
 *     sum_faces C_f (h_nbr - h_c) + q_c = 0,
 * constant-head neighbours go to the right-hand side.  The system is solved
 * by conjugate gradients preconditioned with zero-fill incomplete Cholesky
 * (IC(0)); the unknowns are visited with the layer index fastest because the
 * vertical conductances of thin layers are the strongest couplings.
 * Face flows follow as Q = C (h_upstream_side - h_other_side), signed
 * positive in the +axis direction, so the per-cell imbalance of the returned
 * flows equals the linear-system residual.
 *
 * Build: gcc -O2 -ffp-contract=off -shared -fPIC (no FMA contraction, so the
 * same seed gives the same field on x86_64 and aarch64 hosts).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FG_OK 0
#define FG_ERR_ARG -1
#define FG_ERR_OOM -2
#define FG_ERR_NOCONV -3

static inline size_t nat(int k, int i, int j, int nrow, int ncol) {
    return ((size_t)k * nrow + i) * ncol + j;
}

/* conductance between two cells along one axis; zero if either is inactive */
static inline double cond(double area, double d_a, double k_a, double d_b, double k_b) {
    return 2.0 * area / (d_a / k_a + d_b / k_b);
}

/*
 * Solve for heads and face flows.
 *   K[cells]      hydraulic conductivity (m/s), > 0 where ibound != 0
 *   q_src[cells]  volumetric source (m^3/s; negative = extraction), may be NULL
 *   head[cells]   in: constant-head values at ibound == -1 cells (others ignored)
 *                 out: solved heads (inactive cells: 0)
 *   qx[nlay*nrow*(ncol+1)], qy[nlay*(nrow+1)*ncol], qz[(nlay+1)*nrow*ncol]
 *   tol_abs       stop when max_c |residual_c| <= tol_abs (m^3/s)
 * Returns FG_OK, or FG_ERR_NOCONV if max_iter was reached (flows still written).
 */
int fg_solve(int nlay, int nrow, int ncol,
             const double* delr, const double* delc, const double* dz,
             const double* K, const int8_t* ibound, const double* q_src,
             double* head, double tol_abs, int max_iter,
             double* qx, double* qy, double* qz,
             double* out_maxres, int* out_iters)
{
    if (nlay <= 0 || nrow <= 0 || ncol <= 0) return FG_ERR_ARG;
    const size_t n = (size_t)nlay * nrow * ncol;
    /* solver order: o = (i*ncol + j)*nlay + k */
    const size_t sj = (size_t)nlay, si = (size_t)ncol * nlay;
    double* diag = calloc(n, sizeof(double));
    double* cxm = calloc(n, sizeof(double));   /* coupling to (i, j-1, k) */
    double* cym = calloc(n, sizeof(double));   /* coupling to (i-1, j, k) */
    double* czm = calloc(n, sizeof(double));   /* coupling to (i, j, k-1) */
    double* rhs = calloc(n, sizeof(double));
    double* x = calloc(n, sizeof(double));
    double* r = calloc(n, sizeof(double));
    double* z = calloc(n, sizeof(double));
    double* p = calloc(n, sizeof(double));
    double* ap = calloc(n, sizeof(double));
    double* dinv = calloc(n, sizeof(double));
    uint8_t* unk = calloc(n, 1);
    int rc = FG_OK;
    if (!diag || !cxm || !cym || !czm || !rhs || !x || !r || !z || !p || !ap || !dinv || !unk) {
        rc = FG_ERR_OOM; goto done;
    }
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                size_t c = nat(k, i, j, nrow, ncol);
                unk[o] = ibound[c] > 0;
            }

    /* assemble: for every interior face with two non-inactive cells */
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                size_t c = nat(k, i, j, nrow, ncol);
                if (ibound[c] == 0) continue;
                /* west neighbour */
                if (j > 0) {
                    size_t cn = nat(k, i, j - 1, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delc[i] * dz[k], delr[j - 1], K[cn], delr[j], K[c]);
                        size_t on = o - sj;
                        if (unk[o]) diag[o] += C;
                        if (unk[on]) diag[on] += C;
                        if (unk[o] && unk[on]) cxm[o] = C;
                        else if (unk[o]) rhs[o] += C * head[cn];
                        else if (unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (i > 0) {
                    size_t cn = nat(k, i - 1, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * dz[k], delc[i - 1], K[cn], delc[i], K[c]);
                        size_t on = o - si;
                        if (unk[o]) diag[o] += C;
                        if (unk[on]) diag[on] += C;
                        if (unk[o] && unk[on]) cym[o] = C;
                        else if (unk[o]) rhs[o] += C * head[cn];
                        else if (unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (k > 0) {
                    size_t cn = nat(k - 1, i, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * delc[i], dz[k - 1], K[cn], dz[k], K[c]);
                        size_t on = o - 1;
                        if (unk[o]) diag[o] += C;
                        if (unk[on]) diag[on] += C;
                        if (unk[o] && unk[on]) czm[o] = C;
                        else if (unk[o]) rhs[o] += C * head[cn];
                        else if (unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (unk[o] && q_src) rhs[o] += q_src[c];
            }
    /* isolated unknowns (no conductance at all) are pinned at zero */
    for (size_t o = 0; o < n; o++)
        if (unk[o] && diag[o] == 0.0) unk[o] = 0;

    /* IC(0) pivots: d_o = a_oo - sum_{lower m} a_om^2 / d_m */
    for (size_t o = 0; o < n; o++) {
        if (!unk[o]) { dinv[o] = 0.0; continue; }
        double d = diag[o];
        if (czm[o] != 0.0) d -= czm[o] * czm[o] * dinv[o - 1];
        if (cxm[o] != 0.0) d -= cxm[o] * cxm[o] * dinv[o - sj];
        if (cym[o] != 0.0) d -= cym[o] * cym[o] * dinv[o - si];
        if (!(d > 0.0)) d = diag[o];   /* breakdown guard */
        dinv[o] = 1.0 / d;
    }

    /* initial guess: mean of constant heads, linear in x between them is not assumed */
    {
        double hs = 0.0; size_t nh = 0;
        for (size_t c = 0; c < n; c++) if (ibound[c] < 0) { hs += head[c]; nh++; }
        double h0 = nh ? hs / (double)nh : 0.0;
        for (size_t o = 0; o < n; o++) x[o] = unk[o] ? h0 : 0.0;
    }

#define MATVEC(out, v)                                                          \
    for (size_t o = 0; o < n; o++) {                                            \
        if (!unk[o]) { out[o] = 0.0; continue; }                                \
        double s = diag[o] * v[o];                                              \
        if (czm[o] != 0.0) s -= czm[o] * v[o - 1];                              \
        if (o + 1 < n && czm[o + 1] != 0.0) s -= czm[o + 1] * v[o + 1];         \
        if (cxm[o] != 0.0) s -= cxm[o] * v[o - sj];                             \
        if (o + sj < n && cxm[o + sj] != 0.0) s -= cxm[o + sj] * v[o + sj];     \
        if (cym[o] != 0.0) s -= cym[o] * v[o - si];                             \
        if (o + si < n && cym[o + si] != 0.0) s -= cym[o + si] * v[o + si];     \
        out[o] = s;                                                             \
    }

    MATVEC(ap, x);
    double maxres = 0.0;
    for (size_t o = 0; o < n; o++) {
        r[o] = unk[o] ? rhs[o] - ap[o] : 0.0;
        double a = fabs(r[o]); if (a > maxres) maxres = a;
    }
    int it = 0;
    double rz_old = 0.0;
    while (maxres > tol_abs && it < max_iter) {
        /* z = M^-1 r, M = (D + L) D^-1 (D + U) */
        for (size_t o = 0; o < n; o++) {
            if (!unk[o]) { z[o] = 0.0; continue; }
            double s = r[o];
            if (czm[o] != 0.0) s += czm[o] * z[o - 1];
            if (cxm[o] != 0.0) s += cxm[o] * z[o - sj];
            if (cym[o] != 0.0) s += cym[o] * z[o - si];
            z[o] = s * dinv[o];
        }
        for (size_t oo = n; oo-- > 0;) {
            if (!unk[oo]) continue;
            double s = 0.0;
            if (oo + 1 < n && czm[oo + 1] != 0.0) s += czm[oo + 1] * z[oo + 1];
            if (oo + sj < n && cxm[oo + sj] != 0.0) s += cxm[oo + sj] * z[oo + sj];
            if (oo + si < n && cym[oo + si] != 0.0) s += cym[oo + si] * z[oo + si];
            z[oo] += s * dinv[oo];
        }
        double rz = 0.0;
        for (size_t o = 0; o < n; o++) rz += r[o] * z[o];
        if (it == 0) { for (size_t o = 0; o < n; o++) p[o] = z[o]; }
        else {
            double beta = rz / rz_old;
            for (size_t o = 0; o < n; o++) p[o] = z[o] + beta * p[o];
        }
        rz_old = rz;
        MATVEC(ap, p);
        double pap = 0.0;
        for (size_t o = 0; o < n; o++) pap += p[o] * ap[o];
        if (!(pap > 0.0)) break;
        double alpha = rz / pap;
        maxres = 0.0;
        for (size_t o = 0; o < n; o++) {
            x[o] += alpha * p[o];
            r[o] -= alpha * ap[o];
        }
        it++;
        /* recompute the true residual every 50 iterations to avoid drift */
        if (it % 50 == 0) {
            MATVEC(ap, x);
            for (size_t o = 0; o < n; o++) r[o] = unk[o] ? rhs[o] - ap[o] : 0.0;
        }
        for (size_t o = 0; o < n; o++) { double a = fabs(r[o]); if (a > maxres) maxres = a; }
    }
#undef MATVEC

    /* heads back to natural order */
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                size_t c = nat(k, i, j, nrow, ncol);
                if (ibound[c] > 0) head[c] = unk[o] ? x[o] : 0.0;
                else if (ibound[c] == 0) head[c] = 0.0;
            }

    /* face flows, positive in +axis direction; domain-edge faces carry no flow */
    memset(qx, 0, sizeof(double) * (size_t)nlay * nrow * (ncol + 1));
    memset(qy, 0, sizeof(double) * (size_t)nlay * (nrow + 1) * ncol);
    memset(qz, 0, sizeof(double) * (size_t)(nlay + 1) * nrow * ncol);
    for (int k = 0; k < nlay; k++)
        for (int i = 0; i < nrow; i++)
            for (int j = 0; j < ncol; j++) {
                size_t c = nat(k, i, j, nrow, ncol);
                if (ibound[c] == 0) continue;
                if (j > 0) {
                    size_t cn = nat(k, i, j - 1, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delc[i] * dz[k], delr[j - 1], K[cn], delr[j], K[c]);
                        qx[((size_t)k * nrow + i) * (ncol + 1) + j] = C * (head[cn] - head[c]);
                    }
                }
                if (i > 0) {
                    size_t cn = nat(k, i - 1, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * dz[k], delc[i - 1], K[cn], delc[i], K[c]);
                        qy[((size_t)k * (nrow + 1) + i) * ncol + j] = C * (head[cn] - head[c]);
                    }
                }
                if (k > 0) {
                    size_t cn = nat(k - 1, i, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * delc[i], dz[k - 1], K[cn], dz[k], K[c]);
                        qz[((size_t)k * nrow + i) * ncol + j] = C * (head[cn] - head[c]);
                    }
                }
            }
    if (out_maxres) *out_maxres = maxres;
    if (out_iters) *out_iters = it;
    if (maxres > tol_abs) rc = FG_ERR_NOCONV;
done:
    free(diag); free(cxm); free(cym); free(czm); free(rhs); free(x); free(r);
    free(z); free(p); free(ap); free(dinv); free(unk);
    return rc;
}

/*
 * Per-cell volume balance of a face-flow field: inflow - outflow + q_src,
 * written for every cell with ibound > 0 (others: 0).  Returns max |.|.
 */
double fg_balance(int nlay, int nrow, int ncol, const double* qx, const double* qy,
                  const double* qz, const int8_t* ibound, const double* q_src, double* out)
{
    double mx = 0.0;
    for (int k = 0; k < nlay; k++)
        for (int i = 0; i < nrow; i++)
            for (int j = 0; j < ncol; j++) {
                size_t c = nat(k, i, j, nrow, ncol);
                double b = 0.0;
                if (ibound[c] > 0) {
                    b = qx[((size_t)k * nrow + i) * (ncol + 1) + j]
                      - qx[((size_t)k * nrow + i) * (ncol + 1) + j + 1]
                      + qy[((size_t)k * (nrow + 1) + i) * ncol + j]
                      - qy[((size_t)k * (nrow + 1) + i + 1) * ncol + j]
                      + qz[((size_t)k * nrow + i) * ncol + j]
                      - qz[((size_t)(k + 1) * nrow + i) * ncol + j];
                    if (q_src) b += q_src[c];
                }
                if (out) out[c] = b;
                if (fabs(b) > mx) mx = fabs(b);
            }
    return mx;
}
