/*
 * FP64 CPU oracle of the spline x-ray projector.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or constant with
 * the CUDA library; the two meet only through the seeded input generators.
 *
 * What it computes is the plain definition of the discretised x-ray operator
 * of "Generalized Ray Tracing with Basis Functions for Tomographic
 * Projections" (arXiv 2503.20907):
 *
 *   (H)_{m,k} = phi_{theta_m}( (y_m - <x_k, theta_m^perp>) / h )      Sec. IV.A
 *   forward  p = h * H c,   adjoint  c' = h * H^T p                  Sec. II.B
 *
 * with f = sum_k c_k phi((x - x_k)/h) (eq. def_f, rescaled to spacing h),
 * phi(x1, x2) = beta^n(x1) beta^n(x2) (tensor-product B-spline, Sec. III.C)
 * and phi_theta the x-ray transform of phi (eq. eqproj).  By Prop. 1 with
 * D = 2 (eq. xsa) phi_theta is the 1D convolution of the two rescaled
 * B-splines beta^n(./cos)/|cos| and beta^n(./sin)/|sin|, with a Dirac when a
 * scale is 0.  The convolution integrand is piecewise polynomial of degree
 * 2n, so splitting it at every breakpoint of both factors and applying
 * (n+1)-point Gauss-Legendre on each piece gives the exact integral up to
 * rounding.  No closed form with truncated powers is used: in floating point
 * it cancels catastrophically near the axes.
 *
 * Everything is double precision; inputs given as float are promoted.
 * Sums run in a fixed order (rows j ascending, then i ascending for the
 * forward; rays m ascending for the adjoint), so the brute-force and the
 * row-interval enumerations give bit-identical results.
 *
 * Also here, as independent cross-checks:
 *   - Algorithm 2 (generalized ray tracing, Sec. II.B) with K neighbours
 *     (Lemma 1), used to check that its candidate set covers every nonzero
 *     pair;
 *   - Siddon's classical intersection lengths for pixels (degree 0, Sec. II.A),
 *     an independent algorithm to which the degree-0 projector must reduce.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny;   /* coefficients per row (x1 direction), rows (x2) */
    int32_t degree;   /* spline degree n (tensor-product B-splines) */
    int32_t basis;    /* 0: tensor-product B-spline, 1: 3-direction box-spline */
    double h;         /* grid spacing */
    double cx, cy;    /* grid centre */
} orc_grid;

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */
static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

/* Gauss-Legendre nodes and weights on [-1, 1], q = 1..4 points
 * (roots of the Legendre polynomial P_q; textbook closed forms). */
static void gauss_legendre(int q, double *x, double *w)
{
    if (q == 1) { x[0] = 0.0; w[0] = 2.0; return; }
    if (q == 2) { x[0] = -1.0 / sqrt(3.0); x[1] = -x[0]; w[0] = w[1] = 1.0; return; }
    if (q == 3) {
        x[0] = -sqrt(0.6); x[1] = 0.0; x[2] = sqrt(0.6);
        w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0; return;
    }
    /* q == 4 */
    double r = 2.0 / 7.0 * sqrt(6.0 / 5.0);
    double xa = sqrt(3.0 / 7.0 - r), xb = sqrt(3.0 / 7.0 + r);
    double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    x[0] = -xb; x[1] = -xa; x[2] = xa; x[3] = xb;
    w[0] = wb;  w[1] = wa;  w[2] = wa; w[3] = wb;
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}
static int cmp_double_fwd(const void *a, const void *b) { return cmp_double(a, b); }

/* ------------------------------------------------------------------ */
/* B-spline and footprint                                              */
/* ------------------------------------------------------------------ */

/* Centred B-spline of degree n (support [-(n+1)/2, (n+1)/2]), from the
 * truncated-power definition
 *   beta^n(x) = 1/n! sum_{k=0}^{n+1} (-1)^k C(n+1,k) (x + (n+1)/2 - k)_+^n .
 * Degree 0 takes the midpoint value 1/2 at x = +-1/2. */
double orc_bspline(int n, double x)
{
    int m = n + 1;
    double half = 0.5 * m;
    if (n == 0) {
        double ax = fabs(x);
        return ax < 0.5 ? 1.0 : (ax == 0.5 ? 0.5 : 0.0);
    }
    if (fabs(x) >= half) return 0.0;
    double s = 0.0;
    for (int k = 0; k <= m; ++k) {
        double t = x + half - k;
        if (t <= 0.0) continue;
        double tp = 1.0;
        for (int e = 0; e < n; ++e) tp *= t;
        s += ((k & 1) ? -1.0 : 1.0) * binom(m, k) * tp;
    }
    return s / factorial(n);
}

/* phi_theta(yt) for the unit grid: x-ray transform of beta^n (x) beta^n
 * along direction (ct, st) = (cos theta, sin theta), at offset yt.
 * eq. xsa / Prop. 1: phi_theta = (beta_a * beta_b)(yt), beta_s(t) =
 * beta^n(t/s)/s, a = max(|ct|,|st|), b = min(|ct|,|st|); Dirac when b = 0. */
double orc_footprint(int n, double ct, double st, double yt)
{
    int m = n + 1;
    double a = fmax(fabs(ct), fabs(st));
    double b = fmin(fabs(ct), fabs(st));
    if (b == 0.0) return orc_bspline(n, yt / a) / a;
    double w = 0.5 * m * (a + b);
    if (fabs(yt) >= w) return 0.0;

    /* breakpoints of the integrand in v over the support of beta_b */
    double lo = -0.5 * m * b, hi = 0.5 * m * b;
    double br[2 * 5 + 2];
    int nb = 0;
    for (int k = 0; k <= m; ++k) br[nb++] = b * (k - 0.5 * m);
    for (int k = 0; k <= m; ++k) {
        double v = yt - a * (k - 0.5 * m);
        if (v > lo && v < hi) br[nb++] = v;
    }
    qsort(br, (size_t)nb, sizeof(double), cmp_double);

    double gx[4], gw[4];
    gauss_legendre(m, gx, gw);
    double acc = 0.0;
    for (int p = 0; p + 1 < nb; ++p) {
        double l = br[p], r = br[p + 1];
        if (!(r > l)) continue;
        double mid = 0.5 * (l + r), hw = 0.5 * (r - l);
        double s = 0.0;
        for (int g = 0; g < m; ++g) {
            double v = mid + hw * gx[g];
            s += gw[g] * (orc_bspline(n, (yt - v) / a) / a) * (orc_bspline(n, v / b) / b);
        }
        acc += hw * s;
    }
    return acc;
}

/* ------------------------------------------------------------------ */
/* 3-direction box-spline (Sec. III.D)                                 */
/* ------------------------------------------------------------------ */

/* The box-spline with directions u1 = e1, u2 = e2, u3 = e1 + e2 and
 * centred unit rectangles as factors (Sec. III.D): the density of
 * x = t1 u1 + t2 u2 + t3 u3 with t1, t2, t3 independent and uniform on
 * [-1/2, 1/2].  Given x and t3, (t1, t2) = (x1 - t3, x2 - t3) is fixed (unit
 * Jacobian), so M(x) is the length of the set of t3 in [-1/2, 1/2] with
 * x1 - t3 and x2 - t3 both in [-1/2, 1/2]. */
double orc_box3(double x1, double x2)
{
    double lo = fmax(-0.5, fmax(x1 - 0.5, x2 - 0.5));
    double hi = fmin(0.5, fmin(x1 + 0.5, x2 + 0.5));
    return hi > lo ? hi - lo : 0.0;
}

static int cmp_double_fwd(const void *a, const void *b);

/* phi_theta(yt) for the box-spline: its line integral along direction
 * (ct, st) at offset yt, int M(yt theta^perp + t theta) dt with
 * theta^perp = (st, -ct) (eq. rayparam, eq. eqproj).  M is linear on the
 * triangles cut by the lines x1, x2, x1 - x2 in {-1, 0, 1}, so along the line
 * it is piecewise linear between the crossings of those lines; the
 * trapezoid rule between consecutive crossings is exact. */
double orc_footprint_box(double ct, double st, double yt)
{
    double px = yt * st, py = -yt * ct;     /* a point of the line */
    double tb[16];
    int nt = 0;
    for (int k = -1; k <= 1; ++k) {
        if (ct != 0.0) tb[nt++] = (k - px) / ct;                    /* x1 = k */
        if (st != 0.0) tb[nt++] = (k - py) / st;                    /* x2 = k */
        if (ct != st) tb[nt++] = (k - (px - py)) / (ct - st);       /* x1 - x2 = k */
    }
    qsort(tb, (size_t)nt, sizeof(double), cmp_double_fwd);
    double acc = 0.0;
    for (int i = 0; i + 1 < nt; ++i) {
        double t0 = tb[i], t1 = tb[i + 1];
        if (!(t1 > t0)) continue;
        double m0 = orc_box3(px + t0 * ct, py + t0 * st);
        double m1 = orc_box3(px + t1 * ct, py + t1 * st);
        acc += 0.5 * (t1 - t0) * (m0 + m1);
    }
    return acc;
}

/* Half-width of the support of the box-spline's phi_theta: half the sum of
 * |<theta^perp, u_d>| over the three directions. */
double orc_support_halfwidth_box(double ct, double st)
{
    return 0.5 * (fabs(st) + fabs(ct) + fabs(st - ct));
}

/* Half-width of the support of phi_theta: (n+1)(|cos|+|sin|)/2. */
double orc_support_halfwidth(int n, double ct, double st)
{
    return 0.5 * (n + 1) * (fabs(ct) + fabs(st));
}

/* ------------------------------------------------------------------ */
/* geometry: structured line lists -> (theta, y)                       */
/* ------------------------------------------------------------------ */

/* Parallel beam: line (a, j) has angle ang[a] and offset det0 + j*ddet.
 * Ray index a*n_det + j (angle-major, detector fastest). */
void orc_lines_parallel(int32_t n_ang, const double *ang, int32_t n_det,
                        double det0, double ddet, double *theta, double *y)
{
    for (int32_t a = 0; a < n_ang; ++a)
        for (int32_t j = 0; j < n_det; ++j) {
            theta[(int64_t)a * n_det + j] = ang[a];
            y[(int64_t)a * n_det + j] = det0 + j * ddet;
        }
}

/* Line through points S and D: theta is the direction of D - S and
 * y = <S, theta^perp> with theta^perp = (sin, -cos) (eq. rayparam). */
static void line_from_points(double sx, double sy, double dx, double dy,
                             double *theta, double *y)
{
    double t = atan2(dy - sy, dx - sx);
    *theta = t;
    *y = sx * sin(t) - sy * cos(t);
}

/* Flat-detector fan beam.  Source at dso*(cos b, sin b); detector line
 * through -dod*(cos b, sin b) along u = (-sin b, cos b); bin j centre at
 * offset det0 + j*ddet along u.  Ray index v*n_det + j. */
void orc_lines_fan(int32_t n_view, const double *beta, double dso, double dod,
                   int32_t n_det, double det0, double ddet,
                   double *theta, double *y)
{
    for (int32_t v = 0; v < n_view; ++v) {
        double cb = cos(beta[v]), sb = sin(beta[v]);
        double sx = dso * cb, sy = dso * sb;
        for (int32_t j = 0; j < n_det; ++j) {
            double s = det0 + j * ddet;
            double dx = -dod * cb - s * sb;
            double dy = -dod * sb + s * cb;
            int64_t r = (int64_t)v * n_det + j;
            line_from_points(sx, sy, dx, dy, &theta[r], &y[r]);
        }
    }
}

/* Arbitrary lines through point pairs src[r], dst[r] (each [2]). */
void orc_lines_points(int64_t m, const double *src, const double *dst,
                      double *theta, double *y)
{
    for (int64_t r = 0; r < m; ++r)
        line_from_points(src[2 * r], src[2 * r + 1], dst[2 * r], dst[2 * r + 1],
                         &theta[r], &y[r]);
}

/* ------------------------------------------------------------------ */
/* enumeration of the nonzero pairs of one ray                         */
/* ------------------------------------------------------------------ */

static double node_x1(const orc_grid *g, int32_t i) { return g->cx + (i - 0.5 * (g->nx - 1)) * g->h; }
static double node_x2(const orc_grid *g, int32_t j) { return g->cy + (j - 0.5 * (g->ny - 1)) * g->h; }

/* Offset of the line from node (i, j) in grid units: (y - <x_k, theta^perp>)/h. */
static double offset_yt(const orc_grid *g, double ct, double st, double y, int32_t i, int32_t j)
{
    return (y - (node_x1(g, i) * st - node_x2(g, j) * ct)) / g->h;
}

/* Footprint and support half-width of the grid's basis. */
static double footprint_g(const orc_grid *g, double ct, double st, double yt)
{
    return g->basis == 1 ? orc_footprint_box(ct, st, yt) : orc_footprint(g->degree, ct, st, yt);
}
static double halfwidth_g(const orc_grid *g, double ct, double st)
{
    return g->basis == 1 ? orc_support_halfwidth_box(ct, st) : orc_support_halfwidth(g->degree, ct, st);
}

/* Is (i, j) in the support of the ray?  Open support |yt| < w, except
 * for degree 0 along an axis where the footprint is a rectangle with the
 * midpoint value at its edges, so |yt| <= w. */
static int in_support(int n, double b, double yt, double w)
{
    if (n == 0 && b == 0.0) return fabs(yt) <= w;
    return fabs(yt) < w;
}

/* Column range [i0, i1] that can hold nonzero pairs in row j.  brute != 0
 * returns the whole row; otherwise the interval from |yt(i)| < w, widened
 * by one cell each side (the exact test is applied by the caller). */
static void row_range(const orc_grid *g, double ct, double st, double y, double w,
                      int32_t j, int brute, int32_t *i0, int32_t *i1)
{
    if (brute || fabs(st) < 1e-300) { *i0 = 0; *i1 = g->nx - 1; return; }
    /* yt(i) = (y + x2 ct - x1(i) st)/h, x1(i) = cx + (i - (nx-1)/2) h */
    double ic = ((y + node_x2(g, j) * ct) / st - g->cx) / g->h + 0.5 * (g->nx - 1);
    double half = w / fabs(st);
    double lo = floor(ic - half) - 1.0, hi = ceil(ic + half) + 1.0;
    lo = fmin(fmax(lo, 0.0), (double)g->nx);
    hi = fmax(fmin(hi, (double)(g->nx - 1)), -1.0);
    *i0 = (int32_t)lo;
    *i1 = (int32_t)hi;
}

/* ------------------------------------------------------------------ */
/* forward / adjoint                                                   */
/* ------------------------------------------------------------------ */

static double forward_one(const orc_grid *g, const double *coef, double th, double y, int brute)
{
    int n = g->basis == 1 ? 1 : g->degree;
    double ct = cos(th), st = sin(th);
    double b = fmin(fabs(ct), fabs(st));
    double w = halfwidth_g(g, ct, st);
    double acc = 0.0;
    for (int32_t j = 0; j < g->ny; ++j) {
        int32_t i0, i1;
        row_range(g, ct, st, y, w, j, brute, &i0, &i1);
        for (int32_t i = i0; i <= i1; ++i) {
            double yt = offset_yt(g, ct, st, y, i, j);
            if (!in_support(n, b, yt, w)) continue;
            acc += coef[(int64_t)j * g->nx + i] * footprint_g(g, ct, st, yt);
        }
    }
    return g->h * acc;
}

/* p_m = h * sum_k c_k phi_{theta_m}(yt_{m,k}), m < n_lines. */
void orc_forward(const orc_grid *g, const double *coef, int64_t n_lines,
                 const double *theta, const double *y, double *out,
                 int32_t brute, int32_t n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t r = 0; r < n_lines; ++r)
        out[r] = forward_one(g, coef, theta[r], y[r], brute);
}

/* c'_k = h * sum_m p_m phi_{theta_m}(yt_{m,k}) for the n_pix node indices
 * in pix[] (linear index j*nx + i).  Pixel-driven over all lines, so any
 * subset of nodes can be checked one by one. */
void orc_adjoint_pixels(const orc_grid *g, const double *sino, int64_t n_lines,
                        const double *theta, const double *y,
                        int64_t n_pix, const int64_t *pix, double *out, int32_t n_threads)
{
    int n = g->basis == 1 ? 1 : g->degree;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t q = 0; q < n_pix; ++q) {
        int32_t i = (int32_t)(pix[q] % g->nx), j = (int32_t)(pix[q] / g->nx);
        double acc = 0.0;
        for (int64_t r = 0; r < n_lines; ++r) {
            double ct = cos(theta[r]), st = sin(theta[r]);
            double b = fmin(fabs(ct), fabs(st));
            double w = halfwidth_g(g, ct, st);
            double yt = offset_yt(g, ct, st, y[r], i, j);
            if (!in_support(n, b, yt, w)) continue;
            acc += sino[r] * footprint_g(g, ct, st, yt);
        }
        out[q] = g->h * acc;
    }
}

/* Full adjoint c' = h H^T p over every node. */
void orc_adjoint(const orc_grid *g, const double *sino, int64_t n_lines,
                 const double *theta, const double *y, double *out, int32_t n_threads)
{
    int64_t np = (int64_t)g->nx * g->ny;
    int64_t *pix = (int64_t *)malloc(sizeof(int64_t) * (size_t)np);
    for (int64_t k = 0; k < np; ++k) pix[k] = k;
    orc_adjoint_pixels(g, sino, n_lines, theta, y, np, pix, out, n_threads);
    free(pix);
}

/* Nonzero pairs per line (the visited set V = {(m,k): |yt| < w}).
 * counts[r] receives the number of k for line r; if idx != NULL it also
 * receives the k (ascending j, then i) at idx[offs[r] ...]. */
void orc_visited(const orc_grid *g, int64_t n_lines, const double *theta, const double *y,
                 int32_t brute, int64_t *counts, const int64_t *offs, int64_t *idx,
                 double *min_gap)
{
    int n = g->basis == 1 ? 1 : g->degree;
    double gap = INFINITY;
    for (int64_t r = 0; r < n_lines; ++r) {
        double ct = cos(theta[r]), st = sin(theta[r]);
        double b = fmin(fabs(ct), fabs(st));
        double w = halfwidth_g(g, ct, st);
        int64_t c = 0;
        for (int32_t j = 0; j < g->ny; ++j) {
            int32_t i0, i1;
            row_range(g, ct, st, y[r], w, j, brute, &i0, &i1);
            for (int32_t i = i0; i <= i1; ++i) {
                double yt = offset_yt(g, ct, st, y[r], i, j);
                double d = fabs(fabs(yt) - w);
                if (d < gap) gap = d;
                if (!in_support(n, b, yt, w)) continue;
                if (idx) idx[offs[r] + c] = (int64_t)j * g->nx + i;
                ++c;
            }
        }
        counts[r] = c;
    }
    if (min_gap) *min_gap = gap;
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 with K neighbours (cross-check of Lemma 1)              */
/* ------------------------------------------------------------------ */

/* Candidate set of Algorithm 2 for one line: trace the line through the
 * cells of the grid (cell (p,q) is the square of side h centred on node
 * (p,q)), take each crossed cell and its K neighbours on either side along
 * the minor axis (left/right for mainly vertical lines, |sin| > 1/sqrt 2;
 * up/down otherwise), each cell once.  The trace covers the grid widened
 * by K cells along the minor axis, because a cell outside the grid can be
 * crossed while its neighbours inside still contribute.  mark[] is a
 * caller-owned scratch of nx*ny bytes, zero on entry and on return.
 * Writes the candidate node indices to cand[] and returns their number;
 * *val receives h * sum over candidates of c_k phi(yt) (Algorithm 1). */
int64_t orc_alg2_line(const orc_grid *g, const double *coef, double th, double y,
                      int32_t K, uint8_t *mark, int64_t *cand, double *val)
{
    int n = g->degree;
    double ct = cos(th), st = sin(th);
    int vertical = fabs(st) > fabs(ct);
    /* cell coordinates: node (i,j) is the centre of [i-1/2, i+1/2) x [j-1/2, j+1/2) */
    double ox = g->cx - 0.5 * (g->nx - 1) * g->h, oy = g->cy - 0.5 * (g->ny - 1) * g->h;
    /* a point of the line and its direction, in cell units */
    double px = (y * st - ox) / g->h, py = (-y * ct - oy) / g->h;
    int64_t nc = 0;
    double acc = 0.0;
    int32_t nmaj = vertical ? g->ny : g->nx;
    int32_t nmin = vertical ? g->nx : g->ny;
    /* For every band of the major axis, the crossed cells are those whose
     * minor-axis interval meets the segment of the line inside the band. */
    for (int32_t q = 0; q < nmaj; ++q) {
        double t0, t1;   /* minor coordinate at the two band edges */
        if (vertical) {
            double s0 = (q - 0.5 - py) / st, s1 = (q + 0.5 - py) / st;
            t0 = px + s0 * ct; t1 = px + s1 * ct;
        } else {
            double s0 = (q - 0.5 - px) / ct, s1 = (q + 0.5 - px) / ct;
            t0 = py + s0 * st; t1 = py + s1 * st;
        }
        double tlo = fmin(t0, t1), thi = fmax(t0, t1);
        /* crossed cells p: [p-1/2, p+1/2) meets [tlo, thi] */
        double plo = floor(tlo + 0.5), phi_ = floor(thi + 0.5);
        if (thi + 0.5 == phi_ && phi_ > plo) phi_ -= 1.0;  /* touching an edge only */
        if (phi_ < -K - 1 || plo > nmin + K) continue;
        int32_t a0 = (int32_t)fmax(plo - K, 0.0), a1 = (int32_t)fmin(phi_ + K, (double)(nmin - 1));
        for (int32_t p = a0; p <= a1; ++p) {
            int32_t i = vertical ? p : q, j = vertical ? q : p;
            int64_t k = (int64_t)j * g->nx + i;
            if (mark[k]) continue;
            mark[k] = 1;
            cand[nc++] = k;
            double yt = offset_yt(g, ct, st, y, i, j);
            acc += coef[k] * orc_footprint(n, ct, st, yt);
        }
    }
    for (int64_t c = 0; c < nc; ++c) mark[cand[c]] = 0;
    *val = g->h * acc;
    return nc;
}

/* ------------------------------------------------------------------ */
/* Siddon's method (degree 0)                                          */
/* ------------------------------------------------------------------ */

/* Classical Siddon: intersection lengths of the line with the pixel cells,
 * from the sorted crossings of the line with the grid planes.  Returns
 * sum_k c_k * length_k for the infinite line (theta, y). */
double orc_siddon_line(const orc_grid *g, const double *coef, double th, double y)
{
    double ct = cos(th), st = sin(th);
    double h = g->h;
    double xmin = g->cx - 0.5 * g->nx * h, ymin = g->cy - 0.5 * g->ny * h;
    double xmax = xmin + g->nx * h, ymax = ymin + g->ny * h;
    double px = y * st, py = -y * ct;   /* foot point of the line */
    /* parameter range of the line inside the box */
    double tmin = -INFINITY, tmax = INFINITY;
    if (ct != 0.0) {
        double ta = (xmin - px) / ct, tb = (xmax - px) / ct;
        tmin = fmax(tmin, fmin(ta, tb)); tmax = fmin(tmax, fmax(ta, tb));
    } else if (px < xmin || px > xmax) return 0.0;
    if (st != 0.0) {
        double ta = (ymin - py) / st, tb = (ymax - py) / st;
        tmin = fmax(tmin, fmin(ta, tb)); tmax = fmin(tmax, fmax(ta, tb));
    } else if (py < ymin || py > ymax) return 0.0;
    if (!(tmax > tmin)) return 0.0;
    int cap = g->nx + g->ny + 4;
    double *ts = (double *)malloc(sizeof(double) * (size_t)cap);
    int nt = 0;
    ts[nt++] = tmin;
    if (ct != 0.0)
        for (int i = 0; i <= g->nx; ++i) {
            double t = (xmin + i * h - px) / ct;
            if (t > tmin && t < tmax) ts[nt++] = t;
        }
    if (st != 0.0)
        for (int j = 0; j <= g->ny; ++j) {
            double t = (ymin + j * h - py) / st;
            if (t > tmin && t < tmax) ts[nt++] = t;
        }
    ts[nt++] = tmax;
    qsort(ts, (size_t)nt, sizeof(double), cmp_double);
    double acc = 0.0;
    for (int q = 0; q + 1 < nt; ++q) {
        double len = ts[q + 1] - ts[q];
        if (len <= 0.0) continue;
        double tm = 0.5 * (ts[q] + ts[q + 1]);
        double xm = px + tm * ct, ym = py + tm * st;
        int i = (int)floor((xm - xmin) / h), j = (int)floor((ym - ymin) / h);
        if (i < 0 || i >= g->nx || j < 0 || j >= g->ny) continue;
        acc += coef[(int64_t)j * g->nx + i] * len;
    }
    free(ts);
    return acc;
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
