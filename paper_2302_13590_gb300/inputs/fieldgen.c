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

/* ======================================================================
 * Multigrid-preconditioned CG (used for the large, strongly heterogeneous
 * fields).  Levels store the operator in column order o = (i*nc + j)*nl + k
 * (layer index fastest), so that z-lines are contiguous:
 *   cx[o]: coupling to (i, j-1, k), cy[o]: to (i-1, j, k), cz[o]: to (i, j, k-1)
 * Coarse levels aggregate 2x2x2 cells (Galerkin product with piecewise
 * constant prolongation: coarse couplings are sums of fine couplings across
 * the aggregate faces).  The smoother is z-line Gauss-Seidel over columns in
 * red-black order (forward before, reverse after the coarse correction, so
 * the V-cycle is symmetric and serves as a CG preconditioner); each line is
 * solved exactly with the Thomas algorithm, which takes care of the strong
 * vertical coupling of thin layers.
 * ====================================================================== */

typedef struct {
    int nl, nr, nc;
    size_t n;
    double *diag, *cx, *cy, *cz;
    uint8_t* unk;
    double *x, *b, *r;
} mg_level;

#define MG_MAX_LEVELS 24

static void mg_free_level(mg_level* L)
{
    free(L->diag); free(L->cx); free(L->cy); free(L->cz); free(L->unk);
    free(L->x); free(L->b); free(L->r);
}

static int mg_alloc_level(mg_level* L, int nl, int nr, int nc)
{
    L->nl = nl; L->nr = nr; L->nc = nc;
    L->n = (size_t)nl * nr * nc;
    L->diag = calloc(L->n, sizeof(double)); L->cx = calloc(L->n, sizeof(double));
    L->cy = calloc(L->n, sizeof(double)); L->cz = calloc(L->n, sizeof(double));
    L->unk = calloc(L->n, 1);
    L->x = calloc(L->n, sizeof(double)); L->b = calloc(L->n, sizeof(double)); L->r = calloc(L->n, sizeof(double));
    return (L->diag && L->cx && L->cy && L->cz && L->unk && L->x && L->b && L->r) ? 0 : -1;
}

/* y = A x on one level */
static void mg_apply(const mg_level* L, const double* x, double* y)
{
    const size_t sj = (size_t)L->nl, si = (size_t)L->nc * L->nl, n = L->n;
    for (size_t o = 0; o < n; o++) {
        if (!L->unk[o]) { y[o] = 0.0; continue; }
        double s = L->diag[o] * x[o];
        s -= L->cz[o] * (L->cz[o] != 0.0 ? x[o - 1] : 0.0);
        if (o + 1 < n) s -= L->cz[o + 1] * (L->cz[o + 1] != 0.0 ? x[o + 1] : 0.0);
        s -= L->cx[o] * (L->cx[o] != 0.0 ? x[o - sj] : 0.0);
        if (o + sj < n) s -= L->cx[o + sj] * (L->cx[o + sj] != 0.0 ? x[o + sj] : 0.0);
        s -= L->cy[o] * (L->cy[o] != 0.0 ? x[o - si] : 0.0);
        if (o + si < n) s -= L->cy[o + si] * (L->cy[o + si] != 0.0 ? x[o + si] : 0.0);
        y[o] = s;
    }
}

/* exact solve along the z-line of column (i, j) with the horizontal
 * neighbours held fixed */
static void mg_line(mg_level* L, int i, int j, double* cp, double* dp)
{
    const int nl = L->nl;
    const size_t sj = (size_t)nl, si = (size_t)L->nc * nl, n = L->n;
    const size_t o0 = ((size_t)i * L->nc + j) * nl;
    for (int k = 0; k < nl; k++) {
        size_t o = o0 + k;
        if (!L->unk[o]) { cp[k] = 0.0; dp[k] = 0.0; continue; }
        double rhs = L->b[o];
        if (L->cx[o] != 0.0) rhs += L->cx[o] * L->x[o - sj];
        if (o + sj < n && L->cx[o + sj] != 0.0) rhs += L->cx[o + sj] * L->x[o + sj];
        if (L->cy[o] != 0.0) rhs += L->cy[o] * L->x[o - si];
        if (o + si < n && L->cy[o + si] != 0.0) rhs += L->cy[o + si] * L->x[o + si];
        /* tridiagonal row: -cz[o] x[k-1] + diag x[k] - cz[o+1] x[k+1] = rhs */
        double a = (k > 0) ? -L->cz[o] : 0.0;
        double c = (k + 1 < nl) ? -L->cz[o + 1] : 0.0;
        double den = L->diag[o] - (k > 0 ? a * cp[k - 1] : 0.0);
        cp[k] = c / den;
        dp[k] = (rhs - (k > 0 ? a * dp[k - 1] : 0.0)) / den;
    }
    for (int k = nl - 1; k >= 0; k--) {
        size_t o = o0 + k;
        if (!L->unk[o]) { L->x[o] = 0.0; continue; }
        double v = dp[k] - (k + 1 < nl ? cp[k] * L->x[o + 1] : 0.0);
        L->x[o] = v;
    }
}

static void mg_smooth(mg_level* L, int reverse, double* cp, double* dp)
{
    for (int pass = 0; pass < 2; pass++) {
        int color = reverse ? 1 - pass : pass;
        for (int i = 0; i < L->nr; i++)
            for (int j = 0; j < L->nc; j++)
                if (((i + j) & 1) == color) mg_line(L, i, j, cp, dp);
    }
}

/* build the Galerkin coarse level of F by 2x2x2 aggregation */
static int mg_coarsen(const mg_level* F, mg_level* C)
{
    int cl = F->nl > 1 ? (F->nl + 1) / 2 : 1;
    int cr = F->nr > 1 ? (F->nr + 1) / 2 : 1;
    int cc = F->nc > 1 ? (F->nc + 1) / 2 : 1;
    if (mg_alloc_level(C, cl, cr, cc)) return -1;
    const int nl = F->nl, nc = F->nc;
    for (int i = 0; i < F->nr; i++)
        for (int j = 0; j < F->nc; j++)
            for (int k = 0; k < F->nl; k++) {
                size_t o = ((size_t)i * nc + j) * nl + k;
                if (!F->unk[o]) continue;
                int I = i / 2, J = j / 2, K = k / 2;
                size_t O = ((size_t)I * cc + J) * cl + K;
                C->unk[O] = 1;
                C->diag[O] += F->diag[o];
                if (j > 0 && F->cx[o] != 0.0) {
                    if ((j - 1) / 2 == J) C->diag[O] -= 2.0 * F->cx[o];
                    else C->cx[O] += F->cx[o];
                }
                if (i > 0 && F->cy[o] != 0.0) {
                    if ((i - 1) / 2 == I) C->diag[O] -= 2.0 * F->cy[o];
                    else C->cy[O] += F->cy[o];
                }
                if (k > 0 && F->cz[o] != 0.0) {
                    if ((k - 1) / 2 == K) C->diag[O] -= 2.0 * F->cz[o];
                    else C->cz[O] += F->cz[o];
                }
            }
    for (size_t O = 0; O < C->n; O++)
        if (!C->unk[O]) C->diag[O] = 1.0;
    return 0;
}

static void mg_vcycle(mg_level* lv, int nlev, int l, double* cp, double* dp)
{
    mg_level* L = &lv[l];
    if (l == nlev - 1) {
        for (int s = 0; s < 60; s++) mg_smooth(L, s & 1, cp, dp);
        return;
    }
    mg_smooth(L, 0, cp, dp);
    mg_apply(L, L->x, L->r);
    for (size_t o = 0; o < L->n; o++) L->r[o] = L->unk[o] ? L->b[o] - L->r[o] : 0.0;
    mg_level* C = &lv[l + 1];
    memset(C->b, 0, sizeof(double) * C->n);
    memset(C->x, 0, sizeof(double) * C->n);
    const int cl = C->nl, cc = C->nc;
    for (int i = 0; i < L->nr; i++)
        for (int j = 0; j < L->nc; j++)
            for (int k = 0; k < L->nl; k++) {
                size_t o = ((size_t)i * L->nc + j) * L->nl + k;
                C->b[((size_t)(i / 2) * cc + j / 2) * cl + k / 2] += L->r[o];
            }
    mg_vcycle(lv, nlev, l + 1, cp, dp);
    for (int i = 0; i < L->nr; i++)
        for (int j = 0; j < L->nc; j++)
            for (int k = 0; k < L->nl; k++) {
                size_t o = ((size_t)i * L->nc + j) * L->nl + k;
                if (L->unk[o]) L->x[o] += C->x[((size_t)(i / 2) * cc + j / 2) * cl + k / 2];
            }
    mg_smooth(L, 1, cp, dp);
}

int fg_solve_mg(int nlay, int nrow, int ncol,
                const double* delr, const double* delc, const double* dz,
                const double* K, const int8_t* ibound, const double* q_src,
                double* head, double tol_abs, int max_iter,
                double* qx, double* qy, double* qz,
                double* out_maxres, int* out_iters)
{
    if (nlay <= 0 || nrow <= 0 || ncol <= 0) return FG_ERR_ARG;
    mg_level lv[MG_MAX_LEVELS];
    memset(lv, 0, sizeof(lv));
    int nlev = 0, rc = FG_OK;
    double *xs = NULL, *rs = NULL, *zs = NULL, *ps = NULL, *aps = NULL, *cp = NULL, *dp = NULL;
    if (mg_alloc_level(&lv[0], nlay, nrow, ncol)) { rc = FG_ERR_OOM; goto done; }
    nlev = 1;
    mg_level* L0 = &lv[0];
    const size_t n = L0->n;
    const size_t sj = (size_t)nlay;
    /* assemble the finest level (column order) */
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                L0->unk[o] = ibound[nat(k, i, j, nrow, ncol)] > 0;
            }
    double* rhs = L0->r;   /* temporarily the right-hand side */
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                size_t c = nat(k, i, j, nrow, ncol);
                if (ibound[c] == 0) continue;
                if (j > 0) {
                    size_t cn = nat(k, i, j - 1, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delc[i] * dz[k], delr[j - 1], K[cn], delr[j], K[c]);
                        size_t on = o - sj;
                        if (L0->unk[o]) L0->diag[o] += C;
                        if (L0->unk[on]) L0->diag[on] += C;
                        if (L0->unk[o] && L0->unk[on]) L0->cx[o] = C;
                        else if (L0->unk[o]) rhs[o] += C * head[cn];
                        else if (L0->unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (i > 0) {
                    size_t cn = nat(k, i - 1, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * dz[k], delc[i - 1], K[cn], delc[i], K[c]);
                        size_t on = o - (size_t)ncol * nlay;
                        if (L0->unk[o]) L0->diag[o] += C;
                        if (L0->unk[on]) L0->diag[on] += C;
                        if (L0->unk[o] && L0->unk[on]) L0->cy[o] = C;
                        else if (L0->unk[o]) rhs[o] += C * head[cn];
                        else if (L0->unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (k > 0) {
                    size_t cn = nat(k - 1, i, j, nrow, ncol);
                    if (ibound[cn] != 0) {
                        double C = cond(delr[j] * delc[i], dz[k - 1], K[cn], dz[k], K[c]);
                        size_t on = o - 1;
                        if (L0->unk[o]) L0->diag[o] += C;
                        if (L0->unk[on]) L0->diag[on] += C;
                        if (L0->unk[o] && L0->unk[on]) L0->cz[o] = C;
                        else if (L0->unk[o]) rhs[o] += C * head[cn];
                        else if (L0->unk[on]) rhs[on] += C * head[c];
                    }
                }
                if (L0->unk[o] && q_src) rhs[o] += q_src[c];
            }
    for (size_t o = 0; o < n; o++) {
        if (L0->unk[o] && L0->diag[o] == 0.0) L0->unk[o] = 0;
        if (!L0->unk[o]) L0->diag[o] = 1.0;
    }
    while (nlev < MG_MAX_LEVELS) {
        mg_level* F = &lv[nlev - 1];
        if (F->n <= 64 || (F->nl == 1 && F->nr == 1 && F->nc == 1)) break;
        if (mg_coarsen(F, &lv[nlev])) { rc = FG_ERR_OOM; goto done; }
        nlev++;
    }
    xs = calloc(n, sizeof(double)); rs = calloc(n, sizeof(double)); zs = calloc(n, sizeof(double));
    ps = calloc(n, sizeof(double)); aps = calloc(n, sizeof(double));
    cp = calloc((size_t)nlay + 1, sizeof(double)); dp = calloc((size_t)nlay + 1, sizeof(double));
    if (!xs || !rs || !zs || !ps || !aps || !cp || !dp) { rc = FG_ERR_OOM; goto done; }
    double* b0 = calloc(n, sizeof(double));
    if (!b0) { rc = FG_ERR_OOM; goto done; }
    memcpy(b0, rhs, sizeof(double) * n);
    {
        double hs = 0.0; size_t nh = 0;
        for (size_t c = 0; c < n; c++) if (ibound[c] < 0) { hs += head[c]; nh++; }
        double h0 = nh ? hs / (double)nh : 0.0;
        for (size_t o = 0; o < n; o++) xs[o] = L0->unk[o] ? h0 : 0.0;
    }
    mg_apply(L0, xs, aps);
    double maxres = 0.0;
    for (size_t o = 0; o < n; o++) {
        rs[o] = L0->unk[o] ? b0[o] - aps[o] : 0.0;
        if (fabs(rs[o]) > maxres) maxres = fabs(rs[o]);
    }
    int it = 0;
    double rz_old = 0.0;
    double best = maxres;
    int since_best = 0;
    while (maxres > tol_abs && it < max_iter) {
        /* stop at the rounding floor: no halving of the best residual in 60 iterations */
        if (maxres < 0.5 * best) { best = maxres; since_best = 0; }
        else if (++since_best > 60) break;
        memcpy(L0->b, rs, sizeof(double) * n);
        memset(L0->x, 0, sizeof(double) * n);
        mg_vcycle(lv, nlev, 0, cp, dp);
        memcpy(zs, L0->x, sizeof(double) * n);
        double rz = 0.0;
        for (size_t o = 0; o < n; o++) rz += rs[o] * zs[o];
        if (it == 0) memcpy(ps, zs, sizeof(double) * n);
        else {
            double beta = rz / rz_old;
            for (size_t o = 0; o < n; o++) ps[o] = zs[o] + beta * ps[o];
        }
        rz_old = rz;
        mg_apply(L0, ps, aps);
        double pap = 0.0;
        for (size_t o = 0; o < n; o++) pap += ps[o] * aps[o];
        if (!(pap > 0.0)) break;
        double alpha = rz / pap;
        for (size_t o = 0; o < n; o++) { xs[o] += alpha * ps[o]; rs[o] -= alpha * aps[o]; }
        it++;
        if (it % 20 == 0) {
            mg_apply(L0, xs, aps);
            for (size_t o = 0; o < n; o++) rs[o] = L0->unk[o] ? b0[o] - aps[o] : 0.0;
        }
        maxres = 0.0;
        for (size_t o = 0; o < n; o++) if (fabs(rs[o]) > maxres) maxres = fabs(rs[o]);
    }
    free(b0);
    /* heads back to natural order, then face flows */
    for (int i = 0; i < nrow; i++)
        for (int j = 0; j < ncol; j++)
            for (int k = 0; k < nlay; k++) {
                size_t o = ((size_t)i * ncol + j) * nlay + k;
                size_t c = nat(k, i, j, nrow, ncol);
                if (ibound[c] > 0) head[c] = L0->unk[o] ? xs[o] : 0.0;
                else if (ibound[c] == 0) head[c] = 0.0;
            }
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
    for (int l = 0; l < nlev; l++) mg_free_level(&lv[l]);
    free(xs); free(rs); free(zs); free(ps); free(aps); free(cp); free(dp);
    return rc;
}
