/*
 * wmg_oracle.c -- plain, slow, single-threaded FP64 reference implementation of
 * the wavelet-multigrid (WMG) preconditioned Krylov method for 2D algebraic
 * tomography (Cools, Ghysels, van Aarle, Sijbers, Vanroose, arXiv 1310.0956).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or
 * includes this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg load it. It shares no code, header or table with the GPU
 * path. Every function is written for readability, not speed: the projection
 * matrix W is assembled explicitly (CSR) and applied as two SpMVs, the wavelet
 * operators are applied one 2D Haar step at a time, leaf matrices are factored
 * by dense Cholesky, and the multilevel cycle is the paper's recursion.
 *
 * Geometry (the paper is silent on conventions; these are the readings used):
 *  - image on the unit square [-1/2, 1/2]^2, n x n pixels of width h = 1/n,
 *    stored row-major x[iy*n + ix], iy = 0 at y = -1/2;
 *  - internally all lengths are in pixel units (pixel width 1, image square
 *    [-n/2, n/2]^2); weights are multiplied by h at the end so that w_ij is
 *    the intersection length in unit-square units (Section 2.1, eq. sys);
 *  - ray (a, k) is the line {p : p . (c_a, s_a) = t_k}, t_k = (k-(D-1)/2)*dt + t0
 *    in pixel units, row index i = a*D + k; equispaced angles theta_a = a*pi/m;
 *  - a line lying exactly on a pixel edge gives half of the edge length to each
 *    of the two pixels that share it ("half-split" rule).
 *
 * Parity pins for every function here live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Trigonometric table                                                       */
/* ------------------------------------------------------------------------ */

/* cos/sin of theta = pi*a/m by reduction to the first octant, so that
 * multiples of pi/2 give exact 0/+-1, odd multiples of pi/4 give
 * c = s = sqrt(1/2), and theta, theta+pi/2 receive exactly swapped values. */
static void trig_equispaced(int a, int m, double *c, double *s)
{
    /* theta = (pi/2) * (2a/m) = (pi/2) * (q + r/m), q = quadrant, 0 <= r < m */
    long two_a = 2L * a;
    long q = two_a / m;
    long r = two_a - q * m;
    double cb, sb;                   /* cos, sin of the in-quadrant angle */
    if (r == 0) {
        cb = 1.0; sb = 0.0;
    } else if (2 * r == m) {
        cb = sqrt(0.5); sb = cb;
    } else if (2 * r < m) {
        double phi = (M_PI / 2.0) * ((double)r / (double)m);
        cb = cos(phi); sb = sin(phi);
    } else {
        double phi = (M_PI / 2.0) * ((double)(m - r) / (double)m);
        cb = sin(phi); sb = cos(phi);
    }
    /* rotate by q quarter turns: (c, s) -> (-s, c) */
    for (long i = 0; i < (q & 3); i++) {
        double t = cb;
        cb = -sb; sb = t;
    }
    *c = cb; *s = sb;
}

/* ------------------------------------------------------------------------ */
/* Projection matrix W (Section 2.1)                                         */
/* ------------------------------------------------------------------------ */

typedef struct or_op {
    int n, m, D;
    double dt, t0;
    double *c, *s;        /* m cos / sin */
    int64_t *rowptr;      /* M + 1 */
    int32_t *col;
    double *val;
    int64_t nnz;
} or_op;

/* Growable (col, val) list of one row, merged by column at the end. */
typedef struct { int32_t col; double val; } entry;
typedef struct { entry *e; int64_t len, cap; } rowbuf;

/* Append (j, w); consecutive contributions to the same pixel are merged. */
static void rb_add(rowbuf *rb, int32_t j, double w)
{
    if (w == 0.0) return;
    if (rb->len > 0 && rb->e[rb->len - 1].col == j) { rb->e[rb->len - 1].val += w; return; }
    if (rb->len == rb->cap) {
        rb->cap = rb->cap ? 2 * rb->cap : 64;
        rb->e = realloc(rb->e, (size_t)rb->cap * sizeof(entry));
    }
    rb->e[rb->len].col = j; rb->e[rb->len].val = w; rb->len++;
}

static int cmp_entry(const void *a, const void *b)
{
    int32_t x = ((const entry *)a)->col, y = ((const entry *)b)->col;
    return (x > y) - (x < y);
}

static int cmp_dbl(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Siddon-style parametric walk of one line through the n x n grid (pixel
 * units). Crossings with every vertical and horizontal grid line are merged;
 * each segment between consecutive crossings lies in one pixel (found from the
 * segment midpoint) and contributes its length. Lines on a grid line are the
 * half-split case. */
static void ray_siddon(int n, double c, double s, double T, rowbuf *rb)
{
    const double half = 0.5 * n;
    /* axis-aligned lines: handle exactly, with the half-split rule */
    if (s == 0.0 || c == 0.0) {
        int vertical = (s == 0.0);           /* line X = T/c, or Y = T/s */
        double pos = vertical ? T / c : T / s;
        double u = pos + half;               /* grid coordinate of the line */
        if (u < 0.0 || u > (double)n) return;
        double fl = floor(u);
        for (int i = 0; i < n; i++) {        /* every row (or column) */
            if (u == fl) {                   /* on a grid line: split */
                int lo = (int)fl - 1, hi = (int)fl;
                if (lo >= 0) rb_add(rb, vertical ? i * n + lo : lo * n + i, 0.5);
                if (hi < n) rb_add(rb, vertical ? i * n + hi : hi * n + i, 0.5);
            } else {
                int j = (int)fl;
                rb_add(rb, vertical ? i * n + j : j * n + i, 1.0);
            }
        }
        return;
    }
    /* general line P(l) = T*(c,s) + l*(-s,c) */
    double px = T * c, py = T * s, vx = -s, vy = c;
    /* parameter interval inside the square */
    double lx0 = (-half - px) / vx, lx1 = (half - px) / vx;
    double ly0 = (-half - py) / vy, ly1 = (half - py) / vy;
    double lmin = fmax(fmin(lx0, lx1), fmin(ly0, ly1));
    double lmax = fmin(fmax(lx0, lx1), fmax(ly0, ly1));
    if (!(lmax > lmin)) return;
    double *ls = malloc((size_t)(2 * n + 4) * sizeof(double));
    int cnt = 0;
    ls[cnt++] = lmin;
    ls[cnt++] = lmax;
    for (int i = 0; i <= n; i++) {
        double X = i - half, Y = i - half;
        double l1 = (X - px) / vx, l2 = (Y - py) / vy;
        if (l1 > lmin && l1 < lmax) ls[cnt++] = l1;
        if (l2 > lmin && l2 < lmax) ls[cnt++] = l2;
    }
    qsort(ls, (size_t)cnt, sizeof(double), cmp_dbl);
    for (int q = 0; q + 1 < cnt; q++) {
        double len = ls[q + 1] - ls[q];
        if (len <= 0.0) continue;
        double lm = 0.5 * (ls[q] + ls[q + 1]);
        int ix = (int)floor(px + lm * vx + half);
        int iy = (int)floor(py + lm * vy + half);
        if (ix < 0 || ix >= n || iy < 0 || iy >= n) continue;
        rb_add(rb, iy * n + ix, len);
    }
    free(ls);
}

/* Length of the line {X c + Y s = T} inside the closed box
 * [x0, x0+1] x [y0, y0+1] (Liang-Barsky clipping), with the half-split rule
 * when the line runs along one of the box's edges. */
static double clip_len(double c, double s, double T, double x0, double y0)
{
    if (s == 0.0) {                       /* vertical line X = T/c */
        double X = T / c;
        if (X < x0 || X > x0 + 1.0) return 0.0;
        return (X == x0 || X == x0 + 1.0) ? 0.5 : 1.0;
    }
    if (c == 0.0) {                       /* horizontal line Y = T/s */
        double Y = T / s;
        if (Y < y0 || Y > y0 + 1.0) return 0.0;
        return (Y == y0 || Y == y0 + 1.0) ? 0.5 : 1.0;
    }
    double px = T * c, py = T * s, vx = -s, vy = c;
    double lo = -INFINITY, hi = INFINITY;
    double p[4] = {-vx, vx, -vy, vy};
    double q[4] = {px - x0, x0 + 1.0 - px, py - y0, y0 + 1.0 - py};
    for (int k = 0; k < 4; k++) {
        double r = q[k] / p[k];
        if (p[k] < 0) { if (r > lo) lo = r; }
        else          { if (r < hi) hi = r; }
    }
    return hi > lo ? hi - lo : 0.0;
}

/* Joseph's kernel (Joseph 1982), the paper's choice of W (Section 2.1): the
 * line {x c + y s = T} is sampled where it crosses the centre line of every
 * pixel row (if |c| >= |s|: the line runs closer to the y axis) or every
 * pixel column (otherwise); at each crossing the image is interpolated
 * linearly between the two nearest pixel centres of that row (column), and
 * each sample is weighted by the length of line between consecutive rows
 * (columns), 1 / max(|c|, |s|) pixel widths. Pixels outside the image count as
 * zero. Weights in pixel widths. */
static void ray_joseph(int n, double c, double s, double T, rowbuf *rb)
{
    const double half = 0.5 * n;
    const int by_rows = fabs(c) >= fabs(s);
    const double step = 1.0 / (by_rows ? fabs(c) : fabs(s));
    for (int r = 0; r < n; r++) {
        const double u = r + 0.5 - half;                      /* row y (column x) centre */
        const double v = by_rows ? (T - u * s) / c : (T - u * c) / s;   /* crossing x (y) */
        const double q = v + half - 0.5;                      /* in pixel-centre index units */
        const double f = floor(q);
        const int i0 = (int)f;
        const double w1 = q - f, w0 = 1.0 - w1;
        for (int e = 0; e < 2; e++) {
            const int i = i0 + e;
            const double w = e ? w1 : w0;
            if (i < 0 || i >= n || !(w > 0.0)) continue;
            rb_add(rb, by_rows ? r * n + i : i * n + r, w * step);
        }
    }
}

/* Trapezoid law: chord of a unit pixel at signed distance delta from its
 * centre, for a line with unit normal (c, s). Test-only closed form. */
double or_weight_trapezoid(double c, double s, double delta)
{
    double al = fmax(fabs(c), fabs(s)), be = fmin(fabs(c), fabs(s));
    double d = fabs(delta);
    if (be == 0.0) return d < 0.5 ? 1.0 : (d == 0.5 ? 0.5 : 0.0);
    double L = (0.5 * (al + be) - d) / (al * be);
    if (L < 0.0) L = 0.0;
    if (L > 1.0 / al) L = 1.0 / al;
    return L;
}

or_op *or_op_create(int n, int m, int D, double dt, double t0,
                    const double *angles, int method)
{
    if (n <= 0 || m <= 0 || D <= 0) return NULL;
    or_op *op = calloc(1, sizeof(or_op));
    op->n = n; op->m = m; op->D = D;
    op->dt = dt > 0 ? dt : 1.0; op->t0 = t0;
    op->c = malloc((size_t)m * sizeof(double));
    op->s = malloc((size_t)m * sizeof(double));
    for (int a = 0; a < m; a++) {
        if (angles) { op->c[a] = cos(angles[a]); op->s[a] = sin(angles[a]); }
        else trig_equispaced(a, m, &op->c[a], &op->s[a]);
    }
    const int64_t M = (int64_t)m * D;
    const double h = 1.0 / n;
    op->rowptr = calloc((size_t)M + 1, sizeof(int64_t));
    int64_t cap = 1024, nnz = 0;
    op->col = malloc((size_t)cap * sizeof(int32_t));
    op->val = malloc((size_t)cap * sizeof(double));
    rowbuf rb = {0};
    for (int a = 0; a < m; a++) {
        for (int k = 0; k < D; k++) {
            double T = (k - 0.5 * (D - 1)) * op->dt + op->t0;
            rb.len = 0;
            if (method == 0) {
                ray_siddon(n, op->c[a], op->s[a], T, &rb);
            } else if (method == 2) {
                ray_joseph(n, op->c[a], op->s[a], T, &rb);
            } else {
                for (int iy = 0; iy < n; iy++)
                    for (int ix = 0; ix < n; ix++)
                        rb_add(&rb, iy * n + ix,
                               clip_len(op->c[a], op->s[a], T, ix - 0.5 * n, iy - 0.5 * n));
            }
            /* sort the row by column and merge repeated pixels */
            qsort(rb.e, (size_t)rb.len, sizeof(entry), cmp_entry);
            if (nnz + rb.len > cap) {
                while (nnz + rb.len > cap) cap *= 2;
                op->col = realloc(op->col, (size_t)cap * sizeof(int32_t));
                op->val = realloc(op->val, (size_t)cap * sizeof(double));
            }
            for (int64_t q = 0; q < rb.len; q++) {
                if (q > 0 && rb.e[q].col == rb.e[q - 1].col) {
                    op->val[nnz - 1] += rb.e[q].val * h;
                    continue;
                }
                op->col[nnz] = rb.e[q].col;
                op->val[nnz] = rb.e[q].val * h;
                nnz++;
            }
            op->rowptr[(int64_t)a * D + k + 1] = nnz;
        }
    }
    free(rb.e);
    op->nnz = nnz;
    return op;
}

/* One row (ray (a, k)) of W, built by the same walk as or_op_create without
 * assembling the matrix: for sampled checks at sizes where W does not fit in
 * memory. Entries sorted by column, repeated pixels merged, values in
 * unit-square lengths. Returns the entry count; if it exceeds cap, nothing is
 * written and the negated count is returned. */
int64_t or_ray_row_k(int n, int m, int D, double dt, double t0, const double *angles, int a, int k,
                     int method, int32_t *col, double *val, int64_t cap)
{
    if (n <= 0 || m <= 0 || D <= 0 || a < 0 || a >= m || k < 0 || k >= D) return 0;
    double c, s;
    if (angles) { c = cos(angles[a]); s = sin(angles[a]); }
    else trig_equispaced(a, m, &c, &s);
    dt = dt > 0 ? dt : 1.0;
    const double T = (k - 0.5 * (D - 1)) * dt + t0, h = 1.0 / n;
    rowbuf rb = {0};
    if (method == 2) ray_joseph(n, c, s, T, &rb);
    else ray_siddon(n, c, s, T, &rb);
    qsort(rb.e, (size_t)rb.len, sizeof(entry), cmp_entry);
    int64_t cnt = 0;
    for (int64_t q = 0; q < rb.len; q++)
        if (q == 0 || rb.e[q].col != rb.e[q - 1].col) cnt++;
    if (cnt > cap) { free(rb.e); return -cnt; }
    int64_t w = 0;
    for (int64_t q = 0; q < rb.len; q++) {
        if (q > 0 && rb.e[q].col == rb.e[q - 1].col) { val[w - 1] += rb.e[q].val * h; continue; }
        col[w] = rb.e[q].col;
        val[w] = rb.e[q].val * h;
        w++;
    }
    free(rb.e);
    return cnt;
}

int64_t or_ray_row(int n, int m, int D, double dt, double t0, const double *angles, int a, int k,
                   int32_t *col, double *val, int64_t cap)
{
    return or_ray_row_k(n, m, D, dt, t0, angles, a, k, 0, col, val, cap);
}

void or_op_free(or_op *op)
{
    if (!op) return;
    free(op->c); free(op->s); free(op->rowptr); free(op->col); free(op->val);
    free(op);
}

int64_t or_op_nnz(const or_op *op) { return op->nnz; }

void or_op_export(const or_op *op, int64_t *rowptr, int32_t *col, double *val)
{
    const int64_t M = (int64_t)op->m * op->D;
    memcpy(rowptr, op->rowptr, (size_t)(M + 1) * sizeof(int64_t));
    memcpy(col, op->col, (size_t)op->nnz * sizeof(int32_t));
    memcpy(val, op->val, (size_t)op->nnz * sizeof(double));
}

void or_op_trig(const or_op *op, double *c, double *s)
{
    memcpy(c, op->c, (size_t)op->m * sizeof(double));
    memcpy(s, op->s, (size_t)op->m * sizeof(double));
}

/* Summation order: 0 = natural, 1 = reversed (every SpMV row, the
 * backprojection's row sweep and every dot product run backwards), 2 =
 * pairwise (every SpMV row and every dot product summed by recursive halving;
 * the backprojection's sweep in natural order). Each run gives the same
 * results up to rounding; the differences between the runs measure how much
 * rounding the computed iterates carry. */
static int g_reverse = 0;
void or_set_reverse(int r) { g_reverse = r; }

/* sum of a[i] * b[i] over i < len by recursive halving */
static double pairwise_dot(const double *a, const double *b, int64_t len)
{
    if (len <= 4) {
        double acc = 0.0;
        for (int64_t i = 0; i < len; i++) acc += a[i] * b[i];
        return acc;
    }
    const int64_t h = len / 2;
    return pairwise_dot(a, b, h) + pairwise_dot(a + h, b + h, len - h);
}

/* sum of val[q] * x[col[q]] over q in [q0, q1) by recursive halving */
static double pairwise_row(const or_op *op, const double *x, int64_t q0, int64_t q1)
{
    if (q1 - q0 <= 4) {
        double acc = 0.0;
        for (int64_t q = q0; q < q1; q++) acc += op->val[q] * x[op->col[q]];
        return acc;
    }
    const int64_t h = q0 + (q1 - q0) / 2;
    return pairwise_row(op, x, q0, h) + pairwise_row(op, x, h, q1);
}

/* y = W x  (one SpMV, Section 2.1) */
void or_project(const or_op *op, const double *x, double *y)
{
    const int64_t M = (int64_t)op->m * op->D;
    for (int64_t i = 0; i < M; i++) {
        double acc = 0.0;
        if (g_reverse == 2)
            acc = pairwise_row(op, x, op->rowptr[i], op->rowptr[i + 1]);
        else if (g_reverse)
            for (int64_t q = op->rowptr[i + 1] - 1; q >= op->rowptr[i]; q--)
                acc += op->val[q] * x[op->col[q]];
        else
            for (int64_t q = op->rowptr[i]; q < op->rowptr[i + 1]; q++)
                acc += op->val[q] * x[op->col[q]];
        y[i] = acc;
    }
}

/* x = W^T y  (the transposed SpMV) */
void or_backproject(const or_op *op, const double *y, double *x)
{
    const int64_t M = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    for (int64_t j = 0; j < N; j++) x[j] = 0.0;
    for (int64_t ii = 0; ii < M; ii++) {
        const int64_t i = g_reverse == 1 ? M - 1 - ii : ii;
        for (int64_t q = op->rowptr[i]; q < op->rowptr[i + 1]; q++)
            x[op->col[q]] += op->val[q] * y[i];
    }
}

/* z = (W^T W + lambda I) v  (normal-equation operator, eq. sys_reg) */
static void apply_A(const or_op *op, double lambda, const double *v, double *z, double *tmpM)
{
    const int64_t N = (int64_t)op->n * op->n;
    or_project(op, v, tmpM);
    or_backproject(op, tmpM, z);
    for (int64_t j = 0; j < N; j++) z[j] += lambda * v[j];
}

static double dot(const double *a, const double *b, int64_t len)
{
    double acc = 0.0;
    if (g_reverse == 2)
        return pairwise_dot(a, b, len);
    if (g_reverse)
        for (int64_t i = len - 1; i >= 0; i--) acc += a[i] * b[i];
    else
        for (int64_t i = 0; i < len; i++) acc += a[i] * b[i];
    return acc;
}

/* Relative normal-equation residual ||W^T(b - Wx) - lambda x|| / ||W^T b||. */
double or_ne_residual(const or_op *op, double lambda, const double *b, const double *x)
{
    const int64_t M = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    double *r = malloc((size_t)M * sizeof(double));
    double *g = malloc((size_t)N * sizeof(double));
    double *f = malloc((size_t)N * sizeof(double));
    or_project(op, x, r);
    for (int64_t i = 0; i < M; i++) r[i] = b[i] - r[i];
    or_backproject(op, r, g);
    for (int64_t j = 0; j < N; j++) g[j] -= lambda * x[j];
    or_backproject(op, b, f);
    double res = sqrt(dot(g, g, N)) / sqrt(dot(f, f, N));
    free(r); free(g); free(f);
    return res;
}

/* ------------------------------------------------------------------------ */
/* SIRT (Section 2.2.1, eq. sirt_it)                                         */
/* ------------------------------------------------------------------------ */

/* R = diag(1 / row sums), C = diag(1 / column sums); an empty row or column
 * (a ray missing the image, a pixel no ray crosses) gets 0. */
void or_sirt_scalings(const or_op *op, double *R, double *C)
{
    const int64_t M = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    for (int64_t j = 0; j < N; j++) C[j] = 0.0;
    for (int64_t i = 0; i < M; i++) {
        double rs = 0.0;
        for (int64_t q = op->rowptr[i]; q < op->rowptr[i + 1]; q++) {
            rs += op->val[q];
            C[op->col[q]] += op->val[q];
        }
        R[i] = rs > 0.0 ? 1.0 / rs : 0.0;
    }
    for (int64_t j = 0; j < N; j++) C[j] = C[j] > 0.0 ? 1.0 / C[j] : 0.0;
}

/* x <- x + C (W^T R (b - W x) - lambda x), `iters` times from the given x. */
void or_sirt(const or_op *op, const double *b, double *x, int iters, double lambda,
             double *res_hist)
{
    const int64_t M = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    double *R = malloc((size_t)M * sizeof(double)), *C = malloc((size_t)N * sizeof(double));
    double *r = malloc((size_t)M * sizeof(double)), *g = malloc((size_t)N * sizeof(double));
    or_sirt_scalings(op, R, C);
    if (res_hist) res_hist[0] = or_ne_residual(op, lambda, b, x);
    for (int k = 0; k < iters; k++) {
        or_project(op, x, r);
        for (int64_t i = 0; i < M; i++) r[i] = R[i] * (b[i] - r[i]);
        or_backproject(op, r, g);
        for (int64_t j = 0; j < N; j++) x[j] += C[j] * (g[j] - lambda * x[j]);
        if (res_hist) res_hist[k + 1] = or_ne_residual(op, lambda, b, x);
    }
    free(R); free(C); free(r); free(g);
}

/* ------------------------------------------------------------------------ */
/* Haar operators (Section 2.3.2 eq. intops; Section 3.1.1 eq. intops_wav,    */
/* eq. 1of4 .. 4of4)                                                         */
/* ------------------------------------------------------------------------ */

/* Band ids: LL = 0, LH = 1, HL = 2, HH = 3. With row-major vectorisation the
 * Kronecker factor on the left acts on the row index iy, the right one on ix:
 * LH = I (x) J is low-pass in y and high-pass in x. I = [1 1]/sqrt2 per pair,
 * J = [1 -1]/sqrt2 per pair (even index first). */

/* One analysis step on a side x side grid: out[id] (side/2)^2 = I_id^{2h} in */
static void haar_analysis_step(int side, const double *in, double *out[4])
{
    const int hs = side / 2;
    const double r2 = 1.0 / sqrt(2.0);
    for (int Y = 0; Y < hs; Y++)
        for (int X = 0; X < hs; X++) {
            double v00 = in[(2 * Y) * side + 2 * X], v01 = in[(2 * Y) * side + 2 * X + 1];
            double v10 = in[(2 * Y + 1) * side + 2 * X], v11 = in[(2 * Y + 1) * side + 2 * X + 1];
            /* 1D along x first (rows), then along y */
            double lo0 = r2 * (v00 + v01), hi0 = r2 * (v00 - v01);   /* row 2Y */
            double lo1 = r2 * (v10 + v11), hi1 = r2 * (v10 - v11);   /* row 2Y+1 */
            out[0][Y * hs + X] = r2 * (lo0 + lo1);   /* LL: I in y, I in x */
            out[1][Y * hs + X] = r2 * (hi0 + hi1);   /* LH: I in y, J in x */
            out[2][Y * hs + X] = r2 * (lo0 - lo1);   /* HL: J in y, I in x */
            out[3][Y * hs + X] = r2 * (hi0 - hi1);   /* HH: J in y, J in x */
        }
}

/* One synthesis step: out = sum_id I_{2h,id}^h in[id]  (transpose of above) */
static void haar_synthesis_step(int side, double *const in[4], double *out)
{
    const int hs = side / 2;
    const double r2 = 1.0 / sqrt(2.0);
    for (int Y = 0; Y < hs; Y++)
        for (int X = 0; X < hs; X++) {
            double ll = in[0] ? in[0][Y * hs + X] : 0.0, lh = in[1] ? in[1][Y * hs + X] : 0.0;
            double hl = in[2] ? in[2][Y * hs + X] : 0.0, hh = in[3] ? in[3][Y * hs + X] : 0.0;
            double lo0 = r2 * (ll + hl), lo1 = r2 * (ll - hl);       /* transpose of the y step */
            double hi0 = r2 * (lh + hh), hi1 = r2 * (lh - hh);
            out[(2 * Y) * side + 2 * X] = r2 * (lo0 + hi0);
            out[(2 * Y) * side + 2 * X + 1] = r2 * (lo0 - hi0);
            out[(2 * Y + 1) * side + 2 * X] = r2 * (lo1 + hi1);
            out[(2 * Y + 1) * side + 2 * X + 1] = r2 * (lo1 - hi1);
        }
}

/* Wavelet-packet analysis of an n x n image to depth L: every node of the
 * 4-ary tree is split into its four bands. Output layout: leaf k (path
 * id_1 .. id_L, id_1 = first split, k = sum id_d 4^(L-d)) occupies
 * c[k*nc*nc .. (k+1)*nc*nc) as an nc x nc row-major grid, nc = n / 2^L. */
static void packet_analysis_rec(int side, int depth, int L, const double *in,
                                double *out_leaves)
{
    if (depth == L) { memcpy(out_leaves, in, (size_t)side * side * sizeof(double)); return; }
    const int hs = side / 2;
    const int64_t sub = (int64_t)hs * hs;                 /* size of one child grid */
    int64_t leaves_per_child = 1;
    for (int d = depth + 1; d < L; d++) leaves_per_child *= 4;
    const int nc = side >> (L - depth);
    double *ch[4];
    for (int id = 0; id < 4; id++) ch[id] = malloc((size_t)sub * sizeof(double));
    haar_analysis_step(side, in, ch);
    for (int id = 0; id < 4; id++) {
        packet_analysis_rec(hs, depth + 1, L, ch[id],
                            out_leaves + id * leaves_per_child * (int64_t)nc * nc);
        free(ch[id]);
    }
}

void or_packet_analysis(int n, int L, const double *x, double *c)
{
    packet_analysis_rec(n, 0, L, x, c);
}

static void packet_synthesis_rec(int side, int depth, int L, const double *in_leaves,
                                 double *out)
{
    if (depth == L) { memcpy(out, in_leaves, (size_t)side * side * sizeof(double)); return; }
    const int hs = side / 2;
    const int64_t sub = (int64_t)hs * hs;
    int64_t leaves_per_child = 1;
    for (int d = depth + 1; d < L; d++) leaves_per_child *= 4;
    const int nc = side >> (L - depth);
    double *ch[4];
    for (int id = 0; id < 4; id++) {
        ch[id] = malloc((size_t)sub * sizeof(double));
        packet_synthesis_rec(hs, depth + 1, L,
                             in_leaves + id * leaves_per_child * (int64_t)nc * nc, ch[id]);
    }
    haar_synthesis_step(side, ch, out);
    for (int id = 0; id < 4; id++) free(ch[id]);
}

void or_packet_synthesis(int n, int L, const double *c, double *x)
{
    packet_synthesis_rec(n, 0, L, c, x);
}

/* ------------------------------------------------------------------------ */
/* WMG preconditioner (Section 3.1.2 WTG scheme, Section 3.1.3 WMG V-cycle)  */
/* ------------------------------------------------------------------------ */

typedef struct or_wmg {
    const or_op *op;
    int L, nu1, nu2, cycle, hdepth;
    double omega, lambda;
    int nc;                 /* leaf grid side n / 2^L */
    int64_t K;              /* 4^L leaves */
    double *Dl;             /* K leaf matrices (nc^2 x nc^2), Cholesky factors after setup */
    double *dinv;           /* 1 / (l1 row sums of A) for the smoother (0 where the sum is 0) */
    int status;             /* 0 ok, -4 a leaf matrix is not positive definite */
} or_wmg;

/* In-place Cholesky A = L L^T (lower triangle); returns -1 on a pivot <= 0. */
static int cholesky(double *A, int p)
{
    for (int j = 0; j < p; j++) {
        double d = A[j * p + j];
        for (int q = 0; q < j; q++) d -= A[j * p + q] * A[j * p + q];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        A[j * p + j] = d;
        for (int i = j + 1; i < p; i++) {
            double v = A[i * p + j];
            for (int q = 0; q < j; q++) v -= A[i * p + q] * A[j * p + q];
            A[i * p + j] = v / d;
        }
    }
    return 0;
}

static void chol_solve(const double *Lf, int p, const double *b, double *x)
{
    for (int i = 0; i < p; i++) {                 /* L y = b */
        double v = b[i];
        for (int q = 0; q < i; q++) v -= Lf[i * p + q] * x[q];
        x[i] = v / Lf[i * p + i];
    }
    for (int i = p - 1; i >= 0; i--) {            /* L^T x = y */
        double v = x[i];
        for (int q = i + 1; q < p; q++) v -= Lf[q * p + i] * x[q];
        x[i] = v / Lf[i * p + i];
    }
}

/* Leaf Galerkin matrices D_k = Q_k^T (W^T W + lambda I) Q_k, where Q_k maps
 * leaf k's nc x nc coefficient grid to the image (the product of the
 * prolongations I_{2h,id}^h along the leaf's path). Computed as G_k^T G_k +
 * lambda I with G_k = W Q_k (the paper's tall-skinny W I_{2h,id}^h, Section
 * 3.1.3), row by row of W. Because each Haar step acts on disjoint 2x2
 * groups, a leaf basis function lives on one 2^L x 2^L pixel block; its
 * pattern on that block is obtained by running the synthesis on a single
 * 2^L x 2^L block. */
static void leaf_matrices(or_wmg *M)
{
    const or_op *op = M->op;
    const int n = op->n, L = M->L, B = 1 << L, nc = M->nc;
    const int64_t K = M->K, P = (int64_t)nc * nc, Mrows = (int64_t)op->m * op->D;
    /* pattern[k][ly*B + lx] = value of leaf k's basis function at local pixel */
    double *pattern = malloc((size_t)(K * B * B) * sizeof(double));
    double *unit = calloc((size_t)K, sizeof(double));
    for (int64_t k = 0; k < K; k++) {
        unit[k] = 1.0;
        or_packet_synthesis(B, L, unit, pattern + k * B * B);   /* leaves are 1x1 here */
        unit[k] = 0.0;
    }
    free(unit);
    memset(M->Dl, 0, (size_t)(K * P * P) * sizeof(double));
    double *g = calloc((size_t)(K * P), sizeof(double));        /* G rows for all leaves */
    int32_t *touched = malloc((size_t)P * sizeof(int32_t));
    char *is_t = calloc((size_t)P, 1);
    for (int64_t i = 0; i < Mrows; i++) {
        int nt = 0;
        for (int64_t q = op->rowptr[i]; q < op->rowptr[i + 1]; q++) {
            int j = op->col[q], iy = j / n, ix = j % n;
            int blk = (iy / B) * nc + (ix / B), loc = (iy % B) * B + (ix % B);
            if (!is_t[blk]) { is_t[blk] = 1; touched[nt++] = blk; }
            for (int64_t k = 0; k < K; k++)
                g[k * P + blk] += op->val[q] * pattern[k * B * B + loc];
        }
        for (int64_t k = 0; k < K; k++) {
            double *Dk = M->Dl + k * P * P;
            for (int u = 0; u < nt; u++)
                for (int v = 0; v < nt; v++)
                    Dk[(int64_t)touched[u] * P + touched[v]] +=
                        g[k * P + touched[u]] * g[k * P + touched[v]];
        }
        for (int u = 0; u < nt; u++) {
            is_t[touched[u]] = 0;
            for (int64_t k = 0; k < K; k++) g[k * P + touched[u]] = 0.0;
        }
    }
    for (int64_t k = 0; k < K; k++)
        for (int64_t u = 0; u < P; u++) M->Dl[k * P * P + u * P + u] += M->lambda;
    free(pattern); free(g); free(touched); free(is_t);
}

or_wmg *or_wmg_create(const or_op *op, int levels, int nu1, int nu2, double omega,
                      double lambda, int cycle, int hybrid_depth, int factor)
{
    const int L = levels - 1;
    if (L < 0 || (op->n % (1 << L)) != 0) return NULL;
    or_wmg *M = calloc(1, sizeof(or_wmg));
    M->op = op; M->L = L; M->nu1 = nu1; M->nu2 = nu2; M->omega = omega;
    M->lambda = lambda; M->cycle = cycle; M->hdepth = hybrid_depth;
    M->nc = op->n >> L;
    M->K = (int64_t)1 << (2 * L);
    const int64_t P = (int64_t)M->nc * M->nc, N = (int64_t)op->n * op->n;
    M->Dl = malloc((size_t)(M->K * P * P) * sizeof(double));
    leaf_matrices(M);
    if (factor)
        for (int64_t k = 0; k < M->K; k++)
            if (cholesky(M->Dl + k * P * P, (int)P) != 0) { M->status = -4; break; }
    /* l1-Jacobi diagonal: row sums of |A| = W^T (W 1) + lambda, all entries >= 0 */
    M->dinv = malloc((size_t)N * sizeof(double));
    double *ones = malloc((size_t)N * sizeof(double));
    double *tmp = malloc((size_t)op->m * op->D * sizeof(double));
    for (int64_t j = 0; j < N; j++) ones[j] = 1.0;
    apply_A(op, lambda, ones, M->dinv, tmp);
    for (int64_t j = 0; j < N; j++) M->dinv[j] = M->dinv[j] > 0.0 ? 1.0 / M->dinv[j] : 0.0;
    free(ones); free(tmp);
    return M;
}

int or_wmg_status(const or_wmg *M) { return M->status; }

/* Copy leaf k's matrix (before factoring) or factor (after). */
void or_wmg_leaf_export(const or_wmg *M, int64_t k, double *out)
{
    const int64_t P = (int64_t)M->nc * M->nc;
    memcpy(out, M->Dl + k * P * P, (size_t)(P * P) * sizeof(double));
}

void or_wmg_dinv_export(const or_wmg *M, double *out)
{
    memcpy(out, M->dinv, (size_t)M->op->n * M->op->n * sizeof(double));
}

void or_wmg_free(or_wmg *M)
{
    if (!M) return;
    free(M->Dl); free(M->dinv); free(M);
}

/* A_p v for a node p at depth d with grid side n/2^d: prolongate v to the
 * image along p's path (the other bands zero), apply W^T W + lambda, and
 * restrict back along the same path: Q_p^T A Q_p v. `path[0..d-1]` = ids. */
static void node_operator(const or_wmg *M, int d, const int *path, const double *v,
                          double *out)
{
    const or_op *op = M->op;
    const int n = op->n;
    const int64_t N = (int64_t)n * n;
    double *img = malloc((size_t)N * sizeof(double));
    double *buf = malloc((size_t)N * sizeof(double));
    double *tmpM = malloc((size_t)op->m * op->D * sizeof(double));
    /* prolongate: from depth d up to depth 0 */
    int side = n >> d;
    memcpy(img, v, (size_t)side * side * sizeof(double));
    for (int q = d - 1; q >= 0; q--) {
        double *in[4] = {NULL, NULL, NULL, NULL};
        in[path[q]] = img;
        haar_synthesis_step(side * 2, in, buf);
        side *= 2;
        memcpy(img, buf, (size_t)side * side * sizeof(double));
    }
    apply_A(op, M->lambda, img, buf, tmpM);
    /* restrict: from depth 0 down to depth d along the path */
    side = n;
    double *ch[4];
    for (int id = 0; id < 4; id++) ch[id] = malloc((size_t)(N / 4) * sizeof(double));
    for (int q = 0; q < d; q++) {
        haar_analysis_step(side, buf, ch);
        side /= 2;
        memcpy(buf, ch[path[q]], (size_t)side * side * sizeof(double));
    }
    memcpy(out, buf, (size_t)side * side * sizeof(double));
    for (int id = 0; id < 4; id++) free(ch[id]);
    free(img); free(buf); free(tmpM);
}

/* Coarse correction e_p = T(p, c_p) of the WTG recursion (Section 3.1.2):
 * split c_p into its four bands, correct the LL band first; in the hybrid
 * cycle (above depth hdepth) recompute the node residual once after the LL
 * correction, c_p' = c_p - A_p I_{2h,LL}^h e_LL; then correct LH, HL, HH
 * from c_p'; at the leaves solve D_k e = c exactly (Cholesky). */
static void wtg_correct(const or_wmg *M, int d, int *path, int64_t leaf, const double *cp,
                        double *ep)
{
    const int side = M->op->n >> d;
    if (d == M->L) {
        const int64_t P = (int64_t)M->nc * M->nc;
        chol_solve(M->Dl + leaf * P * P, (int)P, cp, ep);
        return;
    }
    const int hs = side / 2;
    const int64_t sub = (int64_t)hs * hs;
    double *c[4], *e[4];
    for (int id = 0; id < 4; id++) {
        c[id] = malloc((size_t)sub * sizeof(double));
        e[id] = malloc((size_t)sub * sizeof(double));
    }
    haar_analysis_step(side, cp, c);
    if (M->cycle == 3 && d < M->hdepth) {
        /* fully multiplicative WTG (eq. wmg): the bands LL, LH, HL, HH in
         * turn, each corrected from the node residual left by the
         * corrections before it, c_p - A_p sum_{j < id} I_{2h,j}^h e_j */
        double *v = malloc((size_t)side * side * sizeof(double));
        double *w = malloc((size_t)side * side * sizeof(double));
        for (int id = 0; id < 4; id++) {
            if (id > 0) {
                double *in[4] = {NULL, NULL, NULL, NULL};
                for (int j = 0; j < id; j++) in[j] = e[j];
                haar_synthesis_step(side, in, v);
                node_operator(M, d, path, v, w);
                for (int64_t i = 0; i < (int64_t)side * side; i++) w[i] = cp[i] - w[i];
                haar_analysis_step(side, w, c);
            }
            path[d] = id;
            wtg_correct(M, d + 1, path, leaf * 4 + id, c[id], e[id]);
        }
        haar_synthesis_step(side, e, ep);
        free(v); free(w);
        for (int id = 0; id < 4; id++) { free(c[id]); free(e[id]); }
        return;
    }
    path[d] = 0;
    wtg_correct(M, d + 1, path, leaf * 4 + 0, c[0], e[0]);
    if ((M->cycle == 1 || M->cycle == 2) && d < M->hdepth) {
        double *v = malloc((size_t)side * side * sizeof(double));
        double *w = malloc((size_t)side * side * sizeof(double));
        double *in[4] = {e[0], NULL, NULL, NULL};
        haar_synthesis_step(side, in, v);                /* I_{2h,LL}^h e_LL */
        node_operator(M, d, path, v, w);                 /* A_p v */
        for (int64_t i = 0; i < (int64_t)side * side; i++) w[i] = cp[i] - w[i];
        haar_analysis_step(side, w, c);                  /* bands of c_p' */
        free(v); free(w);
    }
    for (int id = 1; id < 4; id++) {
        path[d] = id;
        wtg_correct(M, d + 1, path, leaf * 4 + id, c[id], e[id]);
    }
    haar_synthesis_step(side, e, ep);
    if (M->cycle == 2 && d < M->hdepth) {
        /* symmetric closing step: the LL correction once more, from the
         * residual of the whole node correction, c_p'' = c_p - A_p e_p */
        double *w = malloc((size_t)side * side * sizeof(double));
        node_operator(M, d, path, ep, w);
        for (int64_t i = 0; i < (int64_t)side * side; i++) w[i] = cp[i] - w[i];
        haar_analysis_step(side, w, c);
        path[d] = 0;
        wtg_correct(M, d + 1, path, leaf * 4 + 0, c[0], e[1]);
        double *in[4] = {e[1], NULL, NULL, NULL};
        haar_synthesis_step(side, in, w);
        for (int64_t i = 0; i < (int64_t)side * side; i++) ep[i] += w[i];
        free(w);
    }
    for (int id = 0; id < 4; id++) { free(c[id]); free(e[id]); }
}

/* z = B s: nu1 l1-Jacobi pre-sweeps from z = 0, one WMG coarse correction of
 * the residual, nu2 post-sweeps. With nu1 = nu2 = 0 this is the paper's WMG
 * cycle exactly (no relaxation, Section 3.1.2). */
void or_wmg_apply(const or_wmg *M, const double *s, double *z)
{
    const or_op *op = M->op;
    const int64_t N = (int64_t)op->n * op->n;
    double *r = malloc((size_t)N * sizeof(double)), *e = malloc((size_t)N * sizeof(double));
    double *tmpM = malloc((size_t)op->m * op->D * sizeof(double));
    int path[64];
    for (int64_t j = 0; j < N; j++) z[j] = 0.0;
    for (int it = 0; it < M->nu1; it++) {
        apply_A(op, M->lambda, z, r, tmpM);
        for (int64_t j = 0; j < N; j++) z[j] += M->omega * M->dinv[j] * (s[j] - r[j]);
    }
    apply_A(op, M->lambda, z, r, tmpM);
    for (int64_t j = 0; j < N; j++) r[j] = s[j] - r[j];
    wtg_correct(M, 0, path, 0, r, e);
    for (int64_t j = 0; j < N; j++) z[j] += e[j];
    for (int it = 0; it < M->nu2; it++) {
        apply_A(op, M->lambda, z, r, tmpM);
        for (int64_t j = 0; j < N; j++) z[j] += M->omega * M->dinv[j] * (s[j] - r[j]);
    }
    free(r); free(e); free(tmpM);
}

/* ------------------------------------------------------------------------ */
/* Krylov solvers on the normal equations (Section 2.3.1)                    */
/* ------------------------------------------------------------------------ */

/* CGLS for min ||Wx - b||^2 + lambda ||x||^2, optionally preconditioned by a
 * symmetric positive definite B (WMG): from x0 (the x passed in when use_x0,
 * else 0), r = b - W x0, s = W^T r - lambda x0,
 * z = B s, p = z, gamma = s.z; then per iteration q = W p,
 * delta = ||q||^2 + lambda ||p||^2, alpha = gamma/delta, x += alpha p,
 * r -= alpha q, s = W^T r - lambda x, z = B s, beta = (s.z)/gamma, p = z + beta p.
 * res_hist[k] = ||s_k|| / ||s_0|| (the relative NE residual). Stops when it
 * drops below rtol or after max_iter iterations; returns the count. */
int or_cgls(const or_op *op, const or_wmg *M, double lambda, const double *b, double *x, int use_x0,
            int max_iter, double rtol, double *res_hist)
{
    const int64_t Mr = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    double *r = malloc((size_t)Mr * sizeof(double)), *q = malloc((size_t)Mr * sizeof(double));
    double *s = malloc((size_t)N * sizeof(double)), *z = malloc((size_t)N * sizeof(double));
    double *p = malloc((size_t)N * sizeof(double));
    if (!use_x0)
        for (int64_t j = 0; j < N; j++) x[j] = 0.0;
    or_project(op, x, q);
    for (int64_t i = 0; i < Mr; i++) r[i] = b[i] - q[i];
    or_backproject(op, r, s);
    for (int64_t j = 0; j < N; j++) s[j] -= lambda * x[j];
    if (M) or_wmg_apply(M, s, z); else memcpy(z, s, (size_t)N * sizeof(double));
    memcpy(p, z, (size_t)N * sizeof(double));
    double gamma = dot(s, z, N);
    const double s0 = sqrt(dot(s, s, N));
    if (res_hist) res_hist[0] = 1.0;
    int k = 0;
    if (s0 == 0.0) goto done;
    while (k < max_iter) {
        or_project(op, p, q);
        double delta = dot(q, q, Mr) + lambda * dot(p, p, N);
        if (delta == 0.0) break;
        double alpha = gamma / delta;
        for (int64_t j = 0; j < N; j++) x[j] += alpha * p[j];
        for (int64_t i = 0; i < Mr; i++) r[i] -= alpha * q[i];
        or_backproject(op, r, s);
        for (int64_t j = 0; j < N; j++) s[j] -= lambda * x[j];
        k++;
        double rel = sqrt(dot(s, s, N)) / s0;
        if (res_hist) res_hist[k] = rel;
        if (rel < rtol) break;
        if (M) or_wmg_apply(M, s, z); else memcpy(z, s, (size_t)N * sizeof(double));
        double gnew = dot(s, z, N);
        double beta = gnew / gamma;
        gamma = gnew;
        for (int64_t j = 0; j < N; j++) p[j] = z[j] + beta * p[j];
    }
done:
    free(r); free(q); free(s); free(z); free(p);
    return k;
}

/* Restarted GMRES(restart) with right preconditioning (Section 2.3.1, the
 * paper's experiments use right preconditioning) on A x = f, A = W^T W +
 * lambda I, f = W^T b, from x0 (the x passed in when use_x0, else 0).
 * Arnoldi by modified Gram-Schmidt, Givens rotations for the least-squares
 * problem; at the end of each cycle x += B (V y). res_hist[k] = |g_{k}| /
 * ||r0|| after k Arnoldi steps (the residual estimate; r0 = f - A x0),
 * replaced at each restart by the true relative residual. */
int or_gmres(const or_op *op, const or_wmg *M, double lambda, const double *b, double *x, int use_x0,
             int restart, int max_iter, double rtol, double *res_hist)
{
    const int64_t Mr = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    const int mr = restart;
    double *V = malloc((size_t)(mr + 1) * N * sizeof(double));
    double *H = calloc((size_t)(mr + 1) * mr, sizeof(double));   /* H[i*mr + j] */
    double *cs = malloc((size_t)mr * sizeof(double)), *sn = malloc((size_t)mr * sizeof(double));
    double *g = malloc((size_t)(mr + 1) * sizeof(double)), *y = malloc((size_t)mr * sizeof(double));
    double *f = malloc((size_t)N * sizeof(double)), *w = malloc((size_t)N * sizeof(double));
    double *u = malloc((size_t)N * sizeof(double)), *tmpM = malloc((size_t)Mr * sizeof(double));
    or_backproject(op, b, f);
    if (use_x0) {
        apply_A(op, lambda, x, w, tmpM);
        for (int64_t t = 0; t < N; t++) V[t] = f[t] - w[t];
    } else {
        for (int64_t j = 0; j < N; j++) x[j] = 0.0;
        memcpy(V, f, (size_t)N * sizeof(double));    /* r0 = f since x0 = 0 */
    }
    const double fn = sqrt(dot(V, V, N));
    if (res_hist) res_hist[0] = 1.0;
    int k = 0;
    if (fn == 0.0) goto done;
    double beta = fn;
    while (k < max_iter) {
        for (int64_t j = 0; j < N; j++) V[j] /= beta;
        memset(g, 0, (size_t)(mr + 1) * sizeof(double));
        g[0] = beta;
        int j = 0;
        int converged = 0;
        for (; j < mr && k < max_iter; j++) {
            if (M) or_wmg_apply(M, V + j * N, u); else memcpy(u, V + j * N, (size_t)N * sizeof(double));
            apply_A(op, lambda, u, w, tmpM);
            for (int i = 0; i <= j; i++) {                       /* MGS */
                double hij = dot(w, V + i * N, N);
                H[i * mr + j] = hij;
                for (int64_t t = 0; t < N; t++) w[t] -= hij * V[i * N + t];
            }
            double hn = sqrt(dot(w, w, N));
            H[(j + 1) * mr + j] = hn;
            if (hn != 0.0)
                for (int64_t t = 0; t < N; t++) V[(j + 1) * N + t] = w[t] / hn;
            for (int i = 0; i < j; i++) {                        /* old rotations */
                double a = H[i * mr + j], c2 = H[(i + 1) * mr + j];
                H[i * mr + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * mr + j] = -sn[i] * a + cs[i] * c2;
            }
            double a = H[j * mr + j], c2 = H[(j + 1) * mr + j];
            double rr = hypot(a, c2);
            cs[j] = a / rr; sn[j] = c2 / rr;
            H[j * mr + j] = rr; H[(j + 1) * mr + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k++;
            double rel = fabs(g[j + 1]) / fn;
            if (res_hist) res_hist[k] = rel;
            if (rel < rtol || hn == 0.0) { converged = 1; j++; break; }
        }
        /* y = H^{-1} g (upper triangular j x j) */
        for (int i = j - 1; i >= 0; i--) {
            double v = g[i];
            for (int q = i + 1; q < j; q++) v -= H[i * mr + q] * y[q];
            y[i] = v / H[i * mr + i];
        }
        memset(w, 0, (size_t)N * sizeof(double));
        for (int i = 0; i < j; i++)
            for (int64_t t = 0; t < N; t++) w[t] += y[i] * V[i * N + t];
        if (M) or_wmg_apply(M, w, u); else memcpy(u, w, (size_t)N * sizeof(double));
        for (int64_t t = 0; t < N; t++) x[t] += u[t];
        /* true residual r = f - A x for the restart */
        apply_A(op, lambda, x, w, tmpM);
        for (int64_t t = 0; t < N; t++) V[t] = f[t] - w[t];
        beta = sqrt(dot(V, V, N));
        if (res_hist) res_hist[k] = beta / fn;
        if (converged || beta / fn < rtol || beta == 0.0) break;
    }
done:
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(f); free(w); free(u); free(tmpM);
    return k;
}

/* Right-preconditioned BiCGStab (van der Vorst, 1992) on (W^T W + lambda) x =
 * W^T b from x0 (the x passed in when use_x0, else 0) -- the Krylov solver
 * of the paper's experiments
 * (Section 2.3.1 and Section 4): the shadow residual is r0; per iteration
 *   rho = <rh, r>, beta = (rho / rho_prev)(alpha / omega),
 *   p = r + beta (p - omega v), ph = B p, v = A ph, alpha = rho / <rh, v>,
 *   s = r - alpha v, sh = B s, t = A sh, omega = <t, s> / <t, t>,
 *   x += alpha ph + omega sh, r = s - omega t,
 * with B the WMG cycle (identity when M is NULL). res_hist[k] = |r_k| / |r_0|.
 * *status: 0 converged (rtol) or r = 0, 1 iteration cap, -5 breakdown
 * (rho or <rh, v> zero, or omega zero with r nonzero). Returns the count. */
int or_bicgstab(const or_op *op, const or_wmg *M, double lambda, const double *b, double *x, int use_x0,
                int max_iter, double rtol, double *res_hist, int *status)
{
    const int64_t Mr = (int64_t)op->m * op->D, N = (int64_t)op->n * op->n;
    double *r = malloc((size_t)N * sizeof(double)), *rh = malloc((size_t)N * sizeof(double));
    double *p = calloc((size_t)N, sizeof(double)), *v = calloc((size_t)N, sizeof(double));
    double *ph = malloc((size_t)N * sizeof(double)), *sv = malloc((size_t)N * sizeof(double));
    double *sh = malloc((size_t)N * sizeof(double)), *t = malloc((size_t)N * sizeof(double));
    double *tmpM = malloc((size_t)Mr * sizeof(double));
    or_backproject(op, b, r);                          /* r0 = f - A x0 */
    if (use_x0) {
        apply_A(op, lambda, x, t, tmpM);
        for (int64_t j = 0; j < N; j++) r[j] -= t[j];
    } else {
        for (int64_t j = 0; j < N; j++) x[j] = 0.0;
    }
    memcpy(rh, r, (size_t)N * sizeof(double));
    const double r0 = sqrt(dot(r, r, N));
    if (res_hist) res_hist[0] = 1.0;
    int k = 0, st = 1;
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    if (r0 == 0.0) { st = 0; goto done; }
    while (k < max_iter) {
        const double rho = dot(rh, r, N);
        if (rho == 0.0) { st = -5; break; }
        const double beta = (rho / rho_prev) * (alpha / omega);
        for (int64_t j = 0; j < N; j++) p[j] = r[j] + beta * (p[j] - omega * v[j]);
        if (M) or_wmg_apply(M, p, ph); else memcpy(ph, p, (size_t)N * sizeof(double));
        apply_A(op, lambda, ph, v, tmpM);
        const double rv = dot(rh, v, N);
        if (rv == 0.0) { st = -5; break; }
        alpha = rho / rv;
        for (int64_t j = 0; j < N; j++) sv[j] = r[j] - alpha * v[j];
        if (M) or_wmg_apply(M, sv, sh); else memcpy(sh, sv, (size_t)N * sizeof(double));
        apply_A(op, lambda, sh, t, tmpM);
        const double tt = dot(t, t, N);
        omega = tt > 0.0 ? dot(t, sv, N) / tt : 0.0;
        for (int64_t j = 0; j < N; j++) {
            x[j] += alpha * ph[j] + omega * sh[j];
            r[j] = sv[j] - omega * t[j];
        }
        k++;
        const double rel = sqrt(dot(r, r, N)) / r0;
        if (res_hist) res_hist[k] = rel;
        if (rel < rtol || rel == 0.0) { st = 0; break; }
        if (omega == 0.0) { st = -5; break; }
        rho_prev = rho;
    }
done:
    if (status) *status = st;
    free(r); free(rh); free(p); free(v); free(ph); free(sv); free(sh); free(t); free(tmpM);
    return k;
}
