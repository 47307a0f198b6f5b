/*
 * Sequential fp64 oracle for reduce, scan and reduce-by-index and their
 * reverse-mode derivatives ("Reverse-Mode AD of Reduce-by-Index and Scan in
 * Futhark", arXiv 2310.03568).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; operators are named by
 * this file's own integer codes (ORC_*), which the Python wrapper maps from
 * strings.
 *
 * What it computes, and from which passage:
 *   - forward passes by their sequential definitions:
 *       reduce          : the left fold  e (.) a0 (.) a1 ...          (Sec. 3.1)
 *       scan (inclusive): rs[0] = as[0]; rs[i] = rs[i-1] (.) as[i]   (Sec. 5.1)
 *       reduce_by_index : for i in 0..n-1, if 0 <= k < w,
 *                         hist[k] = hist[k] (.) vs[i]                (Sec. 4)
 *   - vector-Jacobian products by the sequential chain rule: the fold or loop
 *     is unrolled into its statements acc' = acc (.) a and the core rewrite
 *     rule (Eq. 1) is applied to each, last statement first.  For scan this
 *     is exactly the rolled return-sweep loop of Sec. 5.1.  No parallel
 *     rewrite of the paper (Figs 2-7) is used here: those are what the GPU
 *     library implements, and this file is what they are checked against.
 *   - Jacobian-vector products by tangent propagation through the same loops
 *     (used only for dot-product tests <J v, u> = <v, J^T u>).
 *   - the lifted primal residuals the specialised rules save:
 *       reduce (*)      : (number of zeros, product of the non-zeros)  (Fig. 3)
 *       reduce_by_index : the same per bin                           (Sec. 4.2.3)
 *       min / max       : the index of the selected element, lowest index on
 *                         ties, sentinel n for "no element"      (Sec. 3.2.2, Fig. 5)
 *   - a stable sort of [0..n-1] by key (Fig. 4's radixSortByFirst), here a
 *     counting sort, with out-of-range keys placed last.
 *
 * Operators (Fig. 8 for the tuple ones), element arity d:
 *   ADD, MUL, MIN, MAX : scalars (d = 1)
 *   LIN (linFnComp)    : (b, c) meaning x -> b + c*x;
 *                        (b1,c1) (.) (b2,c2) = (b2 + c2*b1, c2*c1)     (d = 2)
 *   MM2 (matMul2x2)    : (a, b, c, d) row-major 2x2; X (.) Y = X * Y   (d = 4)
 *   MM3, MM5           : row-major 3x3 / 5x5 matrices, X (.) Y = X * Y (d = 9, 25)
 *   SOP (sumOfProd)    : (p, s); (p1,s1) (.) (p2,s2) = (p1 + p2 + s1*s2, s1 + s2),
 *                        associative and commutative (Sec. 3.3's example of an
 *                        invertible operator); with elements (0, a_i) the
 *                        reduction gives (sum_{i<j} a_i a_j, sum_i a_i)  (d = 2)
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - min/max ties: the lifted operator of Fig. 5 keeps the smaller index; the
 *     value returned is the one stored at that index.  The initial histogram
 *     hist0 acts as index -1, so it wins ties against every element.
 *   - the derivative of min/max follows the selected index (Sec. 3.2.2).
 *   - keys outside [0, m) are skipped (Sec. 4) and their adjoint is 0 (Fig. 4).
 *
 * Every array is fp64, AoS with the operator's arity; keys are int64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_ADD = 0, ORC_MUL = 1, ORC_MIN = 2, ORC_MAX = 3, ORC_LIN = 4, ORC_MM2 = 5, ORC_SOP = 6,
       ORC_MM3 = 7, ORC_MM5 = 8 };

#define MAXD 25

/* Side of the square matrix operators, 0 for the others. */
static int mat_side(int op) {
    if (op == ORC_MM2) return 2;
    if (op == ORC_MM3) return 3;
    if (op == ORC_MM5) return 5;
    return 0;
}

static int arity(int op) {
    if (op == ORC_LIN || op == ORC_SOP) return 2;
    if (mat_side(op)) return mat_side(op) * mat_side(op);
    return 1;
}

/* Z = X Y for q x q row-major matrices. */
static void mat_product(int q, const double *x, const double *y, double *z) {
    for (int i = 0; i < q; i++)
        for (int j = 0; j < q; j++) {
            double s = 0.0;
            for (int k = 0; k < q; k++) s += x[q * i + k] * y[q * k + j];
            z[q * i + j] = s;
        }
}

int oracle_arity(int op) { return arity(op); }

/* Neutral element e of each operator. */
static void neutral(int op, double *e) {
    switch (op) {
    case ORC_ADD: e[0] = 0.0; break;
    case ORC_MUL: e[0] = 1.0; break;
    case ORC_MIN: e[0] = INFINITY; break;
    case ORC_MAX: e[0] = -INFINITY; break;
    case ORC_LIN: e[0] = 0.0; e[1] = 1.0; break;            /* x -> 0 + 1*x */
    case ORC_MM2:
    case ORC_MM3:
    case ORC_MM5:
        for (int i = 0; i < mat_side(op); i++)
            for (int j = 0; j < mat_side(op); j++) e[mat_side(op) * i + j] = (i == j) ? 1.0 : 0.0;
        break;
    case ORC_SOP: e[0] = 0.0; e[1] = 0.0; break;
    }
}

/*
 * For min/max: does the left operand (value x, index ix) win against the
 * right one (value y, index iy)?  Fig. 5's min^L: the smaller value wins; on
 * equal values the smaller index wins.
 */
static int left_wins(int op, double x, int64_t ix, double y, int64_t iy) {
    if (op == ORC_MIN) {
        if (x < y) return 1;
        if (x > y) return 0;
    } else {
        if (x > y) return 1;
        if (x < y) return 0;
    }
    return ix <= iy;
}

/* z = x (.) y for the non-selecting operators. */
static void combine(int op, const double *x, const double *y, double *z) {
    double t[MAXD];
    switch (op) {
    case ORC_ADD: t[0] = x[0] + y[0]; break;
    case ORC_MUL: t[0] = x[0] * y[0]; break;
    case ORC_LIN:                      /* (b1,c1) (.) (b2,c2) = (b2 + c2*b1, c2*c1) */
        t[0] = y[0] + y[1] * x[0];
        t[1] = y[1] * x[1];
        break;
    case ORC_MM2:                      /* Z[i][j] = sum_k X[i][k] * Y[k][j] */
    case ORC_MM3:
    case ORC_MM5:
        mat_product(mat_side(op), x, y, t);
        break;
    case ORC_SOP:                      /* (p1,s1) (.) (p2,s2) = (p1 + p2 + s1*s2, s1 + s2) */
        t[0] = x[0] + y[0] + x[1] * y[1];
        t[1] = x[1] + y[1];
        break;
    }
    memcpy(z, t, sizeof(double) * arity(op));
}

/*
 * Eq. 1 applied to z = x (.) y with adjoint zb: xb = dz/dx^T zb, yb = dz/dy^T zb
 * (both SET, not accumulated).  For min/max, xwins says which operand was
 * selected.
 */
static void combine_vjp(int op, const double *x, const double *y, int xwins,
                        const double *zb, double *xb, double *yb) {
    switch (op) {
    case ORC_ADD: xb[0] = zb[0]; yb[0] = zb[0]; break;
    case ORC_MUL: xb[0] = y[0] * zb[0]; yb[0] = x[0] * zb[0]; break;
    case ORC_MIN:
    case ORC_MAX:
        xb[0] = xwins ? zb[0] : 0.0;
        yb[0] = xwins ? 0.0 : zb[0];
        break;
    case ORC_LIN:
        /* z0 = y0 + y1*x0, z1 = y1*x1 */
        xb[0] = y[1] * zb[0];
        xb[1] = y[1] * zb[1];
        yb[0] = zb[0];
        yb[1] = x[0] * zb[0] + x[1] * zb[1];
        break;
    case ORC_MM2:
    case ORC_MM3:
    case ORC_MM5: {
        /* Z = X Y:  Xb[i][k] = sum_j Zb[i][j] Y[k][j];  Yb[k][j] = sum_i X[i][k] Zb[i][j] */
        const int q = mat_side(op);
        for (int i = 0; i < q; i++)
            for (int k = 0; k < q; k++) {
                double s = 0.0;
                for (int j = 0; j < q; j++) s += zb[q * i + j] * y[q * k + j];
                xb[q * i + k] = s;
            }
        for (int k = 0; k < q; k++)
            for (int j = 0; j < q; j++) {
                double s = 0.0;
                for (int i = 0; i < q; i++) s += x[q * i + k] * zb[q * i + j];
                yb[q * k + j] = s;
            }
        break;
    }
    case ORC_SOP:
        /* z0 = x0 + y0 + x1*y1, z1 = x1 + y1 */
        xb[0] = zb[0];
        xb[1] = y[1] * zb[0] + zb[1];
        yb[0] = zb[0];
        yb[1] = x[1] * zb[0] + zb[1];
        break;
    }
}

/* Tangent of z = x (.) y: zd = dz/dx xd + dz/dy yd. */
static void combine_jvp(int op, const double *x, const double *y, int xwins,
                        const double *xd, const double *yd, double *zd) {
    double t[MAXD];
    switch (op) {
    case ORC_ADD: t[0] = xd[0] + yd[0]; break;
    case ORC_MUL: t[0] = xd[0] * y[0] + x[0] * yd[0]; break;
    case ORC_MIN:
    case ORC_MAX: t[0] = xwins ? xd[0] : yd[0]; break;
    case ORC_LIN:
        t[0] = yd[0] + yd[1] * x[0] + y[1] * xd[0];
        t[1] = yd[1] * x[1] + y[1] * xd[1];
        break;
    case ORC_MM2:
    case ORC_MM3:
    case ORC_MM5: {
        const int q = mat_side(op);
        for (int i = 0; i < q; i++)
            for (int j = 0; j < q; j++) {
                double s = 0.0;
                for (int k = 0; k < q; k++)
                    s += xd[q * i + k] * y[q * k + j] + x[q * i + k] * yd[q * k + j];
                t[q * i + j] = s;
            }
        break;
    }
    case ORC_SOP:
        t[0] = xd[0] + yd[0] + xd[1] * y[1] + x[1] * yd[1];
        t[1] = xd[1] + yd[1];
        break;
    }
    memcpy(zd, t, sizeof(double) * arity(op));
}

static int is_select(int op) { return op == ORC_MIN || op == ORC_MAX; }

/* ------------------------------------------------------------------------ */
/* reduce (Sec. 3)                                                           */
/* ------------------------------------------------------------------------ */

/*
 * y = e (.) a0 (.) ... (.) a_{n-1}, folded left to right.  For min/max, idx
 * receives the index of the selected element (n if none: empty input, or
 * every element loses to the neutral element -- impossible for finite data).
 * The neutral element carries index n, the largest, so any element equal to
 * it wins the tie, as Fig. 5's neutral (n, inf) prescribes.
 */
void oracle_reduce_fwd(int op, int64_t n, const double *x, double *y, int64_t *idx) {
    int d = arity(op);
    double acc[MAXD];
    int64_t iacc = n;
    neutral(op, acc);
    for (int64_t i = 0; i < n; i++) {
        if (is_select(op)) {
            if (!left_wins(op, acc[0], iacc, x[i], i)) { acc[0] = x[i]; iacc = i; }
        } else {
            combine(op, acc, x + i * d, acc);
        }
    }
    memcpy(y, acc, sizeof(double) * d);
    if (idx) *idx = iacc;
}

/*
 * xbar = (dy/dx)^T ybar by the return sweep of the fold: record the
 * accumulator before every step, then apply Eq. 1 to each step
 * acc_{i+1} = acc_i (.) a_i from the last one back.
 */
void oracle_reduce_vjp(int op, int64_t n, const double *x, const double *ybar, double *xbar) {
    int d = arity(op);
    double *trace = (double *)malloc(sizeof(double) * d * (size_t)(n > 0 ? n : 1));
    int64_t *itrace = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double acc[MAXD], accb[MAXD], xb[MAXD], yb[MAXD];
    int64_t iacc = n;
    neutral(op, acc);
    for (int64_t i = 0; i < n; i++) {
        memcpy(trace + i * d, acc, sizeof(double) * d);
        itrace[i] = iacc;
        if (is_select(op)) {
            if (!left_wins(op, acc[0], iacc, x[i], i)) { acc[0] = x[i]; iacc = i; }
        } else {
            combine(op, acc, x + i * d, acc);
        }
    }
    memcpy(accb, ybar, sizeof(double) * d);
    for (int64_t i = n - 1; i >= 0; i--) {
        int xw = is_select(op) ? left_wins(op, trace[i], itrace[i], x[i], i) : 0;
        combine_vjp(op, trace + i * d, x + i * d, xw, accb, xb, yb);
        memcpy(xbar + i * d, yb, sizeof(double) * d);
        memcpy(accb, xb, sizeof(double) * d);
    }
    free(trace);
    free(itrace);
}

/* ydot = (dy/dx) xdot by tangent propagation through the fold. */
void oracle_reduce_jvp(int op, int64_t n, const double *x, const double *xdot, double *ydot) {
    int d = arity(op);
    double acc[MAXD], accd[MAXD];
    int64_t iacc = n;
    neutral(op, acc);
    for (int k = 0; k < d; k++) accd[k] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        if (is_select(op)) {
            int xw = left_wins(op, acc[0], iacc, x[i], i);
            combine_jvp(op, acc, x + i, xw, accd, xdot + i, accd);
            if (!xw) { acc[0] = x[i]; iacc = i; }
        } else {
            combine_jvp(op, acc, x + i * d, 0, accd, xdot + i * d, accd);
            combine(op, acc, x + i * d, acc);
        }
    }
    memcpy(ydot, accd, sizeof(double) * d);
}

/* Fig. 3's lifted primal: number of exact zeros and product of the non-zeros. */
void oracle_reduce_mul_lifted(int64_t n, const double *x, int64_t *nzero, double *prod_nonzero) {
    int64_t z = 0;
    double p = 1.0;
    for (int64_t i = 0; i < n; i++) {
        if (x[i] == 0.0) z++;
        else p *= x[i];
    }
    *nzero = z;
    *prod_nonzero = p;
}

/* ------------------------------------------------------------------------ */
/* scan (Sec. 5)                                                             */
/* ------------------------------------------------------------------------ */

/*
 * For min/max scans: does the running result rs[i-1] win against as[i]?  The
 * running result always comes from an earlier index, so it wins ties (Fig. 5's
 * lifted operator, lowest index first).
 */
static int scan_left_wins(int op, const double *prev, const double *xi, int64_t i) {
    return left_wins(op, prev[0], i - 1, xi[0], i);
}

/* Inclusive scan by the loop of Sec. 5.1: rs[0] = as[0]; rs[i] = rs[i-1] (.) as[i]. */
void oracle_scan_fwd(int op, int64_t n, const double *x, double *y) {
    int d = arity(op);
    if (n <= 0) return;
    memcpy(y, x, sizeof(double) * d);
    for (int64_t i = 1; i < n; i++) {
        if (is_select(op)) y[i] = scan_left_wins(op, y + i - 1, x + i, i) ? y[i - 1] : x[i];
        else combine(op, y + (i - 1) * d, x + i * d, y + i * d);
    }
}

/*
 * The rolled return sweep of Sec. 5.1:
 *   rb = copy ybar
 *   for i = n-1 .. 1:  rb[i-1] += d(rs[i-1] (.) as[i])/d rs[i-1] * rb[i]
 *                      ab[i]    = d(rs[i-1] (.) as[i])/d as[i]   * rb[i]
 *   ab[0] = rb[0]
 * For min/max the step's derivative follows the selected operand (the
 * earlier one on ties).  rbar, when not NULL, receives the final rb: the
 * adjoint of each scan result rs[i] (lambda_i).
 */
void oracle_scan_vjp_rbar(int op, int64_t n, const double *x, const double *ybar, double *xbar,
                          double *rbar) {
    int d = arity(op);
    if (n <= 0) return;
    double *rs = (double *)malloc(sizeof(double) * d * (size_t)n);
    double *rb = (double *)malloc(sizeof(double) * d * (size_t)n);
    double xb[MAXD], yb[MAXD];
    oracle_scan_fwd(op, n, x, rs);
    memcpy(rb, ybar, sizeof(double) * d * (size_t)n);
    for (int64_t i = n - 1; i >= 1; i--) {
        const int xw = is_select(op) ? scan_left_wins(op, rs + i - 1, x + i, i) : 0;
        combine_vjp(op, rs + (i - 1) * d, x + i * d, xw, rb + i * d, xb, yb);
        for (int k = 0; k < d; k++) rb[(i - 1) * d + k] += xb[k];
        memcpy(xbar + i * d, yb, sizeof(double) * d);
    }
    memcpy(xbar, rb, sizeof(double) * d);
    if (rbar) memcpy(rbar, rb, sizeof(double) * d * (size_t)n);
    free(rs);
    free(rb);
}

void oracle_scan_vjp(int op, int64_t n, const double *x, const double *ybar, double *xbar) {
    oracle_scan_vjp_rbar(op, n, x, ybar, xbar, NULL);
}

/* Tangent propagation through the scan loop. */
void oracle_scan_jvp(int op, int64_t n, const double *x, const double *xdot, double *ydot) {
    int d = arity(op);
    if (n <= 0) return;
    double *rs = (double *)malloc(sizeof(double) * d * (size_t)n);
    oracle_scan_fwd(op, n, x, rs);
    memcpy(ydot, xdot, sizeof(double) * d);
    for (int64_t i = 1; i < n; i++) {
        const int xw = is_select(op) ? scan_left_wins(op, rs + i - 1, x + i, i) : 0;
        combine_jvp(op, rs + (i - 1) * d, x + i * d, xw, ydot + (i - 1) * d, xdot + i * d, ydot + i * d);
    }
    free(rs);
}

/* ------------------------------------------------------------------------ */
/* reduce_by_index (Sec. 4)                                                  */
/* ------------------------------------------------------------------------ */

/*
 * The sequential definition of Sec. 4, starting from hist0 (or from e when
 * hist0 is NULL).  For min/max, idx[j] receives the index of the selected
 * element of bin j, or n when the bin is empty or hist0[j] won (hist0 acts as
 * index -1).
 */
void oracle_hist_fwd(int op, int64_t n, int64_t m, const int64_t *keys, const double *vals,
                     const double *hist0, double *hist, int64_t *idx) {
    int d = arity(op);
    int64_t *ih = NULL;
    for (int64_t j = 0; j < m; j++) {
        if (hist0) memcpy(hist + j * d, hist0 + j * d, sizeof(double) * d);
        else neutral(op, hist + j * d);
    }
    if (is_select(op)) {
        ih = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t j = 0; j < m; j++) ih[j] = hist0 ? -1 : n;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) continue;
        if (is_select(op)) {
            if (!left_wins(op, hist[k], ih[k], vals[i], i)) { hist[k] = vals[i]; ih[k] = i; }
        } else {
            combine(op, hist + k * d, vals + i * d, hist + k * d);
        }
    }
    if (idx && is_select(op))
        for (int64_t j = 0; j < m; j++) idx[j] = ih[j] < 0 ? n : ih[j];
    free(ih);
}

/*
 * valsbar and hist0bar (either may be NULL) by the return sweep of the
 * sequential loop: one accumulator per bin, hist0 (or e) as its initial value;
 * Eq. 1 is applied to every executed statement hist[k] = hist[k] (.) vs[i],
 * last one first.  Elements with out-of-range keys get adjoint 0.
 */
void oracle_hist_vjp(int op, int64_t n, int64_t m, const int64_t *keys, const double *vals,
                     const double *hist0, const double *histbar, double *valsbar, double *hist0bar) {
    int d = arity(op);
    double *h = (double *)malloc(sizeof(double) * d * (size_t)(m > 0 ? m : 1));
    double *hb = (double *)malloc(sizeof(double) * d * (size_t)(m > 0 ? m : 1));
    double *trace = (double *)malloc(sizeof(double) * d * (size_t)(n > 0 ? n : 1));
    int64_t *ih = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *itrace = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double xb[MAXD], yb[MAXD];
    for (int64_t j = 0; j < m; j++) {
        if (hist0) memcpy(h + j * d, hist0 + j * d, sizeof(double) * d);
        else neutral(op, h + j * d);
        ih[j] = hist0 ? -1 : n;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) continue;
        memcpy(trace + i * d, h + k * d, sizeof(double) * d);
        itrace[i] = ih[k];
        if (is_select(op)) {
            if (!left_wins(op, h[k], ih[k], vals[i], i)) { h[k] = vals[i]; ih[k] = i; }
        } else {
            combine(op, h + k * d, vals + i * d, h + k * d);
        }
    }
    memcpy(hb, histbar, sizeof(double) * d * (size_t)m);
    for (int64_t i = n - 1; i >= 0; i--) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) {
            if (valsbar)
                for (int c = 0; c < d; c++) valsbar[i * d + c] = 0.0;
            continue;
        }
        int xw = is_select(op) ? left_wins(op, trace[i], itrace[i], vals[i], i) : 0;
        combine_vjp(op, trace + i * d, vals + i * d, xw, hb + k * d, xb, yb);
        if (valsbar) memcpy(valsbar + i * d, yb, sizeof(double) * d);
        memcpy(hb + k * d, xb, sizeof(double) * d);
    }
    if (hist0bar) memcpy(hist0bar, hb, sizeof(double) * d * (size_t)m);
    free(h);
    free(hb);
    free(trace);
    free(ih);
    free(itrace);
}

/* Tangent propagation through the sequential loop (hist0dot may be NULL). */
void oracle_hist_jvp(int op, int64_t n, int64_t m, const int64_t *keys, const double *vals,
                     const double *hist0, const double *valsdot, const double *hist0dot,
                     double *histdot) {
    int d = arity(op);
    double *h = (double *)malloc(sizeof(double) * d * (size_t)(m > 0 ? m : 1));
    int64_t *ih = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; j++) {
        if (hist0) memcpy(h + j * d, hist0 + j * d, sizeof(double) * d);
        else neutral(op, h + j * d);
        ih[j] = hist0 ? -1 : n;
        for (int c = 0; c < d; c++) histdot[j * d + c] = hist0dot ? hist0dot[j * d + c] : 0.0;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) continue;
        if (is_select(op)) {
            int xw = left_wins(op, h[k], ih[k], vals[i], i);
            combine_jvp(op, h + k, vals + i, xw, histdot + k, valsdot + i, histdot + k);
            if (!xw) { h[k] = vals[i]; ih[k] = i; }
        } else {
            combine_jvp(op, h + k * d, vals + i * d, 0, histdot + k * d, valsdot + i * d, histdot + k * d);
            combine(op, h + k * d, vals + i * d, h + k * d);
        }
    }
    free(h);
    free(ih);
}

/* Sec. 4.2.3's lifted primal per bin: zero count and product of the non-zeros. */
void oracle_hist_mul_lifted(int64_t n, int64_t m, const int64_t *keys, const double *vals,
                            int64_t *nzero, double *prod_nonzero) {
    for (int64_t j = 0; j < m; j++) { nzero[j] = 0; prod_nonzero[j] = 1.0; }
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) continue;
        if (vals[i] == 0.0) nzero[k]++;
        else prod_nonzero[k] *= vals[i];
    }
}

/*
 * Stable sort of [0..n-1] by key (Fig. 4, radixSortByFirst): a counting sort.
 * Keys outside [0, m) are treated as the key m, i.e. they come last, in index
 * order.
 */
void oracle_sort_perm(int64_t n, int64_t m, const int64_t *keys, int64_t *perm) {
    int64_t *count = (int64_t *)calloc((size_t)(m + 2), sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) k = m;
        count[k + 1]++;
    }
    for (int64_t j = 0; j <= m; j++) count[j + 1] += count[j];
    for (int64_t i = 0; i < n; i++) {
        int64_t k = keys[i];
        if (k < 0 || k >= m) k = m;
        perm[count[k]++] = i;
    }
    free(count);
}
