/*
 * Plain FP64 CPU oracle for the PeriDEM hot path (bond-based peridynamics with
 * critical-stretch breaking, nodal contact, rigid planar walls, velocity-Verlet).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library; the CUDA library never does, and
 * the two share no code.  It is deliberately slow and obvious: every quantity
 * is computed from its definition in caller node order, in double precision,
 * with no blocking, fusion or reordering.  Build with -O2 -ffp-contract=off
 * (no FMA contraction, no fast-math) so that the bond and contact predicates
 * are evaluated exactly as written.
 *
 * Citations are to the paper's sections and equations:
 *   Sec. 3.1, Eq. (peri), Eq. (pmb), stretch definition    -> bond force
 *   Sec. 3.1.1, Table "peri-combined", bond memory gamma,
 *   Eq. (peri-damage)                                      -> breaking, damage
 *   Sec. 3.2, Eq. (repulsive-force)                        -> inter-grain contact
 *   Sec. 3.3, Eq. (damping-force)                          -> normal contact damping
 *   Sec. 3.3, Eq. (regularized-friction)                   -> stick-slip friction
 *   Sec. 5 "Self-contact forces", Eq. (peri-damage-self)    -> same-grain contact
 *   Sec. 4.1 "Contact between peridynamic body and wall"    -> wall force
 *   Sec. 4.1.1 "Contact with multiple wall boundaries"      -> inclusion-exclusion
 *   Sec. 3.5 Eq. (motion), Sec. 5.2 velocity-Verlet        -> time integration
 *   Sec. 5.3.1 / 5.3.2                                     -> bond removal filters
 *   Sec. 1 (split-off particles), no algorithm given        -> fragments
 * Readings of gaps and errata are stated at each function.
 *
 * Parity status: every function below is pinned by tests under tests/
 * (closed forms, invariants, brute force, textbook special cases), except the
 * post-damage fracture trajectory, which is chaotic: "parity unpinned" beyond
 * step-by-step comparison from a shared state.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* error bits returned by the force evaluation */
#define ORC_ERR_NONFINITE 1
#define ORC_ERR_WALL 2

/* filter kinds (Sec. 5.3) */
#define ORC_FILTER_NOTCH 1
#define ORC_FILTER_SPHERE 2

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the OpenMP build (the timed CPU baseline on all host cores); the
 * serial build ignores it and reports 1. */
int orc_set_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Material constants.                                                       */
/* ------------------------------------------------------------------------- */
/*
 * Bond-based PD fixes Poisson's ratio at 1/4 in 3-D (end of Sec. 3.1.1), so the
 * bulk modulus is K = E / (3 (1 - 2 nu)) = 2E/3.
 *
 * constants == 0 (default): the self-consistent constant-micromodulus values
 *   c  = 18 K / (pi delta^4)     (bulk strain energy matched, see tests)
 *   s0 = sqrt(5 G0 / (9 K delta)) (crack energy matched, see tests)
 * constants == 1: the values printed in the paper's table (3-D, constant row)
 *   c  = 12 E / (pi delta^4 (1 - nu)),  s0 = sqrt(5 pi G0 / (12 E delta)).
 * Reading: the printed pair is 4/3 and sqrt(pi/2) times the self-consistent
 * pair; it is kept only behind the switch.
 * Contact stiffness (Sec. 3.2): K_n = 18 K / (pi delta^5) times a factor f_c,
 * i.e. K_n = f_c c / delta with the default c.
 * micromodulus == 1: the conic micromodulus of the table, c(|xi|) = c (delta - |xi|);
 * c is then the coefficient.  Self-consistent values (same two energy matches):
 *   c  = 90 K / (pi delta^5),  s0 = sqrt(2 G0 / (3 K delta));
 * printed (constants == 1): c = 60 E / (pi delta^5 (1 - nu)), s0 = sqrt(7 pi G0 / (12 E delta)).
 */
void orc_constants(double E, double G0, double delta, double contact_factor, int constants, int micromodulus,
                   double out[4] /* K, c, s0, Kn */)
{
    const double nu = 0.25;
    double K = E / (3.0 * (1.0 - 2.0 * nu));
    double c, s0;
    if (micromodulus == 1 && constants == 1) {
        c = 60.0 * E / (ORC_PI * pow(delta, 5) * (1.0 - nu));
        s0 = sqrt(7.0 * ORC_PI * G0 / (12.0 * E * delta));
    } else if (micromodulus == 1) {
        c = 90.0 * K / (ORC_PI * pow(delta, 5));
        s0 = sqrt(2.0 * G0 / (3.0 * K * delta));
    } else if (constants == 1) {
        c = 12.0 * E / (ORC_PI * pow(delta, 4) * (1.0 - nu));
        s0 = sqrt(5.0 * ORC_PI * G0 / (12.0 * E * delta));
    } else {
        c = 18.0 * K / (ORC_PI * pow(delta, 4));
        s0 = sqrt(5.0 * G0 / (9.0 * K * delta));
    }
    double Kn = contact_factor * 18.0 * K / (ORC_PI * pow(delta, 5));
    out[0] = K;
    out[1] = c;
    out[2] = s0;
    out[3] = Kn;
}

/* ------------------------------------------------------------------------- */
/* Bond family (Sec. 3.1: H_eps(x) intersected with the grain P_i).          */
/* ------------------------------------------------------------------------- */
static double sq3(double a, double b, double c) { return ((a * a) + (b * b)) + (c * c); }

/*
 * Bond removal filters of Sec. 5.3.  The endpoints are passed in canonical
 * order (smaller caller index first) so that both directions of a bond get
 * the same decision.
 *  - notch (Sec. 5.3.1): the segment x1 + t (x2 - x1) meets the plane
 *    a x + b y + c z + d = 0 at t = -(a x1 + b y1 + c z1 + d) / (a dx + b dy + c dz);
 *    the bond is dropped when 0 < t < 1.  Reading: the paper's plane is
 *    unbounded; the crossing point must also lie in the notch face, given as an
 *    axis-aligned box [p[4..6], p[7..9]].
 *  - inner sphere (Sec. 5.3.2): dropped when either end lies strictly inside
 *    the sphere (cases 1 and 2 of the paper).
 */
static int orc_filter_drops(const double *x1, const double *x2, int nf, const int32_t *kinds,
                            const double *prm)
{
    for (int f = 0; f < nf; ++f) {
        const double *p = prm + 12 * f;
        if (kinds[f] == ORC_FILTER_NOTCH) {
            double dx = x2[0] - x1[0], dy = x2[1] - x1[1], dz = x2[2] - x1[2];
            double num = ((p[0] * x1[0] + p[1] * x1[1]) + p[2] * x1[2]) + p[3];
            double den = (p[0] * dx + p[1] * dy) + p[2] * dz;
            if (den != 0.0) {
                double t = -num / den;
                if (t > 0.0 && t < 1.0) {
                    double r0 = x1[0] + t * dx, r1 = x1[1] + t * dy, r2 = x1[2] + t * dz;
                    if (r0 >= p[4] && r0 <= p[7] && r1 >= p[5] && r1 <= p[8] && r2 >= p[6] &&
                        r2 <= p[9])
                        return 1;
                }
            }
        } else if (kinds[f] == ORC_FILTER_SPHERE) {
            double R2 = p[3] * p[3];
            double d1 = sq3(x1[0] - p[0], x1[1] - p[1], x1[2] - p[2]);
            double d2 = sq3(x2[0] - p[0], x2[1] - p[1], x2[2] - p[2]);
            if (d1 < R2 || d2 < R2) return 1;
        }
    }
    return 0;
}

/* Is j a bond partner of i?  Same grain and |x_j - x_i| < delta strictly
 * (Eq. pmb: the force vanishes for |xi| >= eps), minus the filters. */
static int orc_is_bond(const double *x, const int32_t *grain, double delta2, int64_t i, int64_t j,
                       int nf, const int32_t *kinds, const double *prm)
{
    if (i == j || grain[i] != grain[j]) return 0;
    const double *a = x + 3 * i, *b = x + 3 * j;
    double r2 = sq3(b[0] - a[0], b[1] - a[1], b[2] - a[2]);
    if (!(r2 < delta2)) return 0;
    if (nf > 0) {
        if (i < j) return !orc_filter_drops(a, b, nf, kinds, prm);
        return !orc_filter_drops(b, a, nf, kinds, prm);
    }
    return 1;
}

/* Row i of the bond list by brute force over all nodes, ascending j. */
int64_t orc_bond_row(int64_t n, const double *x, const int32_t *grain, double delta, int nf,
                     const int32_t *kinds, const double *prm, int64_t i, int32_t *out)
{
    double delta2 = delta * delta;
    int64_t k = 0;
    for (int64_t j = 0; j < n; ++j)
        if (orc_is_bond(x, grain, delta2, i, j, nf, kinds, prm)) {
            if (out) out[k] = (int32_t)j;
            ++k;
        }
    return k;
}

/* Whole bond list by brute force, O(n^2).  rowptr has n+1 entries; col may be
 * NULL to count only.  Returns the number of directed bonds. */
int64_t orc_bonds_brute(int64_t n, const double *x, const int32_t *grain, double delta, int nf,
                        const int32_t *kinds, const double *prm, int64_t *rowptr, int32_t *col)
{
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr) rowptr[i] = total;
        total += orc_bond_row(n, x, grain, delta, nf, kinds, prm, i, col ? col + total : NULL);
    }
    if (rowptr) rowptr[n] = total;
    return total;
}

/* ------------------------------------------------------------------------- */
/* A plain uniform cell list: nodes sorted by linear cell key; a neighbour    */
/* query walks the 27 surrounding cells.  It only prunes pairs that are       */
/* certainly out of range (cell size >= cutoff); tests pin it to brute force. */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    double lo[3], cs;
    int64_t dim[3];
    int64_t *key;   /* sorted keys */
    int64_t *idx;   /* node index for each sorted key */
} orc_grid;

typedef struct { int64_t key, idx; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *p = (const orc_kv *)a, *q = (const orc_kv *)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

static void orc_cell_of(const orc_grid *g, const double *p, int64_t c[3])
{
    for (int k = 0; k < 3; ++k) {
        int64_t v = (int64_t)floor((p[k] - g->lo[k]) / g->cs);
        if (v < 0) v = 0;
        if (v >= g->dim[k]) v = g->dim[k] - 1;
        c[k] = v;
    }
}

static int orc_grid_build(orc_grid *g, int64_t n, const double *p, double cutoff)
{
    g->n = n;
    g->cs = cutoff * (1.0 + 1e-9);
    double hi[3];
    for (int k = 0; k < 3; ++k) { g->lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            if (p[3 * i + k] < g->lo[k]) g->lo[k] = p[3 * i + k];
            if (p[3 * i + k] > hi[k]) hi[k] = p[3 * i + k];
        }
    for (int k = 0; k < 3; ++k) {
        if (n == 0) { g->lo[k] = 0; hi[k] = 0; }
        g->dim[k] = (int64_t)floor((hi[k] - g->lo[k]) / g->cs) + 1;
    }
    orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (size_t)(n > 0 ? n : 1));
    g->key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    g->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!kv || !g->key || !g->idx) { free(kv); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        orc_cell_of(g, p + 3 * i, c);
        kv[i].key = (c[2] * g->dim[1] + c[1]) * g->dim[0] + c[0];
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    for (int64_t i = 0; i < n; ++i) { g->key[i] = kv[i].key; g->idx[i] = kv[i].idx; }
    free(kv);
    return 0;
}

static void orc_grid_free(orc_grid *g) { free(g->key); free(g->idx); }

static int64_t orc_lower_bound(const int64_t *a, int64_t n, int64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

static int orc_cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

/* Every node of the 27 cells around point q (it may include nodes beyond the
 * cutoff; callers apply the exact predicate), written to buf (capacity n) in
 * ascending index order; returns the count. */
static int64_t orc_grid_near(const orc_grid *g, const double *q, int64_t *buf)
{
    int64_t c[3], m = 0;
    orc_cell_of(g, q, c);
    for (int64_t dz = -1; dz <= 1; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
                if (cx < 0 || cy < 0 || cz < 0 || cx >= g->dim[0] || cy >= g->dim[1] ||
                    cz >= g->dim[2])
                    continue;
                int64_t key = (cz * g->dim[1] + cy) * g->dim[0] + cx;
                int64_t s = orc_lower_bound(g->key, g->n, key);
                for (int64_t t = s; t < g->n && g->key[t] == key; ++t) buf[m++] = g->idx[t];
            }
    qsort(buf, (size_t)m, sizeof(int64_t), orc_cmp_i64);
    return m;
}

/* Bond list through the cell list (cell size = delta); same predicate. */
int64_t orc_bonds_cells(int64_t n, const double *x, const int32_t *grain, double delta, int nf,
                        const int32_t *kinds, const double *prm, int64_t *rowptr, int32_t *col)
{
    orc_grid g;
    if (orc_grid_build(&g, n, x, delta) != 0) return -1;
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double delta2 = delta * delta;
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr) rowptr[i] = total;
        int64_t m = orc_grid_near(&g, x + 3 * i, buf);
        for (int64_t t = 0; t < m; ++t) {
            int64_t j = buf[t];
            if (orc_is_bond(x, grain, delta2, i, j, nf, kinds, prm)) {
                if (col) col[total] = (int32_t)j;
                ++total;
            }
        }
    }
    if (rowptr) rowptr[n] = total;
    free(buf);
    orc_grid_free(&g);
    return total;
}

/* ------------------------------------------------------------------------- */
/* Ball cut by orthogonal planes (Sec. 4.1.1, contact with several walls).   */
/* ------------------------------------------------------------------------- */
/*
 * In an orthonormal frame (X, Y, Z) centred on the node, the region of the
 * ball |r| < R that lies beyond the planes X = a, Y = b and Z = c is
 *   W(a, b, c) = { r : |r| < R, X > a, Y > b, Z > c }.
 * A wall whose outward axis is X and which lies at distance d from the node
 * cuts off W(d, -R, -R), its spherical cap; two orthogonal walls share
 * W(d1, d2, -R) and three mutually orthogonal walls W(d1, d2, d3).  The paper
 * gives no formula for the shared regions; here their volume and first moments
 * are the iterated integrals of the definition, evaluated by adaptive Simpson
 * quadrature: over Z, then over Y, with the X extent of W at (Y, Z) in closed
 * form.  Every integrand is continuous; the quadrature splits each interval at
 * the points where the integrand's formula changes.
 */
typedef struct { double R, a, b, s2; int what; } orc_wctx; /* s2: R^2 - Z^2 at the current Z */

/* X extent of W at (Y, Z): the chord {X > a, X^2 < w^2}, w^2 = s2 - Y^2;
 * what = 0: its length; 1: its X moment; 2: Y times its length */
static double orc_chord(const orc_wctx *q, double Y)
{
    double w2 = q->s2 - Y * Y;
    if (!(w2 > 0.0)) return 0.0;
    double w = sqrt(w2);
    double lo = q->a > -w ? q->a : -w;
    if (!(lo < w)) return 0.0;
    if (q->what == 0) return w - lo;
    if (q->what == 1) return 0.5 * (w * w - lo * lo);
    return Y * (w - lo);
}

typedef double (*orc_fn)(const void *, double);

static double orc_simpson_rec(orc_fn f, const void *ctx, double x0, double x1, double f0, double fm, double f1,
                              double whole, double eps, int depth)
{
    double m = 0.5 * (x0 + x1), l = 0.5 * (x0 + m), r = 0.5 * (m + x1);
    double fl = f(ctx, l), fr = f(ctx, r);
    double left = (m - x0) / 6.0 * (f0 + 4.0 * fl + fm), right = (x1 - m) / 6.0 * (fm + 4.0 * fr + f1);
    double both = left + right;
    if (depth <= 0 || fabs(both - whole) <= 15.0 * eps) return both + (both - whole) / 15.0;
    return orc_simpson_rec(f, ctx, x0, m, f0, fl, fm, left, 0.5 * eps, depth - 1) +
           orc_simpson_rec(f, ctx, m, x1, fm, fr, f1, right, 0.5 * eps, depth - 1);
}

/* adaptive Simpson over [x0, x1] split at the sorted break points inside it */
static double orc_integrate(orc_fn f, const void *ctx, double x0, double x1, const double *brk, int nb, double eps)
{
    double pts[8];
    int np = 0;
    pts[np++] = x0;
    for (int k = 0; k < nb; ++k)
        if (brk[k] > pts[np - 1] && brk[k] < x1) pts[np++] = brk[k];
    pts[np++] = x1;
    double sum = 0.0;
    for (int k = 0; k + 1 < np; ++k) {
        double u = pts[k], v = pts[k + 1];
        if (!(v > u)) continue;
        double fu = f(ctx, u), fv = f(ctx, v), fm = f(ctx, 0.5 * (u + v));
        double whole = (v - u) / 6.0 * (fu + 4.0 * fm + fv);
        sum += orc_simpson_rec(f, ctx, u, v, fu, fm, fv, whole, eps, 40);
    }
    return sum;
}

static double orc_inner(const void *c, double Y) { return orc_chord((const orc_wctx *)c, Y); }

/* integral over Y > b of the chord quantity at the current Z */
static double orc_slice(orc_wctx *q)
{
    if (!(q->s2 > 0.0)) return 0.0;
    double s = sqrt(q->s2);
    double y0 = q->b > -s ? q->b : -s;
    if (!(y0 < s)) return 0.0;
    double brk[2];
    int nb = 0;
    if (q->a * q->a < q->s2) { /* the chord's lower end switches from -w to a at w = |a| */
        double yk = sqrt(q->s2 - q->a * q->a);
        brk[nb++] = -yk;
        brk[nb++] = yk;
    }
    return orc_integrate(orc_inner, q, y0, s, brk, nb, 1e-13 * q->R * q->R);
}

typedef struct { orc_wctx w; double c; int zmom; } orc_octx;

static double orc_outer(const void *c, double Z)
{
    orc_octx *o = (orc_octx *)c;
    orc_wctx q = o->w;
    q.s2 = q.R * q.R - Z * Z;
    double v = orc_slice(&q);
    return o->zmom ? Z * v : v;
}

/* Without the Z plane (c <= -R) the slice of W at fixed Y is the disk of
 * radius r = sqrt(R^2 - Y^2) in (X, Z) beyond the chord X = a: the textbook
 * circular segment, area r^2 acos(a/r) - a sqrt(r^2 - a^2) and X moment
 * (2/3)(r^2 - a^2)^(3/2) for |a| < r (empty for a >= r, the whole disk, area
 * pi r^2 and X moment 0, for a <= -r).  what = 0: area; 1: X moment; 2: Y area. */
static double orc_segment(const void *c, double Y)
{
    const orc_wctx *q = (const orc_wctx *)c;
    double r2 = q->R * q->R - Y * Y;
    if (!(r2 > 0.0)) return 0.0;
    double r = sqrt(r2), a = q->a, area, mx;
    if (a >= r) return 0.0;
    if (a <= -r) { area = ORC_PI * r2; mx = 0.0; }
    else {
        double h = sqrt(r2 - a * a);
        area = r2 * acos(a / r) - a * h;
        mx = (2.0 / 3.0) * h * h * h;
    }
    if (q->what == 0) return area;
    if (q->what == 1) return mx;
    return Y * area;
}

/* volume and first moments (about the node, along X, Y, Z) of W(a, b, c) */
void orc_ball_cut(double R, double a, double b, double c, double out[4])
{
    double z0 = c > -R ? c : -R;
    for (int k = 0; k < 4; ++k) out[k] = 0.0;
    if (!(z0 < R)) return;
    if (c <= -R) {
        double y0 = b > -R ? b : -R, brk[2];
        int nb = 0;
        if (a * a < R * R) { brk[0] = -sqrt(R * R - a * a); brk[1] = -brk[0]; nb = 2; }
        for (int k = 0; k < 3; ++k) {
            orc_wctx q;
            q.R = R; q.a = a; q.b = b; q.s2 = 0.0; q.what = k;
            out[k] = orc_integrate(orc_segment, &q, y0, R, brk, nb, 1e-15 * R * R * R);
        }
        return;
    }
    /* break points in Z where the slice changes form: R^2 - Z^2 = a^2, b^2, a^2 + b^2 */
    double brk[6];
    int nb = 0;
    double t[3] = {a * a, b * b, a * a + b * b};
    for (int k = 0; k < 3; ++k)
        if (t[k] < R * R) {
            double zk = sqrt(R * R - t[k]);
            brk[nb++] = -zk;
            brk[nb++] = zk;
        }
    /* insertion sort of the break points */
    for (int i = 1; i < nb; ++i)
        for (int j = i; j > 0 && brk[j - 1] > brk[j]; --j) { double s = brk[j]; brk[j] = brk[j - 1]; brk[j - 1] = s; }
    double eps = 1e-12 * R * R * R;
    for (int k = 0; k < 4; ++k) {
        orc_octx o;
        o.w.R = R; o.w.a = a; o.w.b = b; o.w.s2 = 0.0;
        o.w.what = k == 1 ? 1 : (k == 2 ? 2 : 0);
        o.c = c;
        o.zmom = k == 3;
        out[k] = orc_integrate(orc_outer, &o, z0, R, brk, nb, eps);
    }
}

/* ------------------------------------------------------------------------- */
/* The problem description shared by the force, step and energy routines.   */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    const double *x;        /* n*3 reference positions */
    const double *vol;      /* n nodal volumes */
    const int32_t *grain;   /* n grain ids */
    const int64_t *rowptr;  /* n+1 */
    const int32_t *col;     /* B, ascending within each row */
    double c, s0, Kn, Rc, rho;
    int break_mode;         /* 0: s > s0 ; 1: |s| > s0 */
    int contact;            /* 0 disables nodal contact */
    int nw;
    const double *walls;    /* nw*9: inward normal, point at t=0, velocity */
    double b[3];            /* body force density, N/m^3 */
    int frozen;             /* 1: evaluate with the given bond memory, no new breaking */
    double beta_d;          /* normal damping coefficient (Sec. 3.3), N s / m^7; 0 = none */
    int conic;              /* 1: conic micromodulus c (delta - |xi|) */
    double delta;           /* horizon (used by the conic micromodulus) */
    double mu;              /* friction coefficient (Sec. 3.3, stick-slip friction); 0 = none */
    double dt_f;            /* time step the friction's stick branch sees; 0 = the Coulomb limit */
    int wall_overlap;       /* 1: inclusion-exclusion over orthogonal walls (Sec. 4.1.1) */
} orc_problem;

/* micromodulus of a bond of reference length L: c, or c (delta - L) when conic */
static double orc_cw(const orc_problem *P, double L) { return P->conic ? P->c * (P->delta - L) : P->c; }

/* slot of j in row i (binary search on the ascending row), or -1 */
static int64_t orc_slot(const orc_problem *P, int64_t i, int64_t j)
{
    int64_t lo = P->rowptr[i], hi = P->rowptr[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if ((int64_t)P->col[mid] < j) lo = mid + 1; else hi = mid;
    }
    if (lo < P->rowptr[i + 1] && (int64_t)P->col[lo] == j) return lo;
    return -1;
}

/*
 * Contact partners of node i at positions p = x + u (Sec. 3.2 and the
 * self-contact section): every j != i with |p_j - p_i| < R_c, except a node of
 * the same grain that still has an intact bond with i (the bond itself then
 * carries the interaction; Eq. peri-damage-self weights self-contact by
 * 1 - gamma).  Written to out (ascending j); returns the count.
 */
static int64_t orc_contacts_of(const orc_problem *P, const double *p, const uint8_t *broken,
                               const orc_grid *g, int64_t i, int64_t *buf, int64_t *out)
{
    double R2 = P->Rc * P->Rc;
    int64_t m = g ? orc_grid_near(g, p + 3 * i, buf) : 0, k = 0;
    int64_t cnt = g ? m : P->n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t j = g ? buf[t] : t;
        if (j == i) continue;
        double d2 = sq3(p[3 * j] - p[3 * i], p[3 * j + 1] - p[3 * i + 1], p[3 * j + 2] - p[3 * i + 2]);
        if (!(d2 < R2)) continue;
        if (P->grain[i] == P->grain[j]) {
            int64_t s = orc_slot(P, i, j);
            if (s >= 0 && !broken[s]) continue;
        }
        out[k++] = j;
    }
    return k;
}

/* All contact pairs (i, j), i != j, both orders, at displacement u; pairs[2k],
 * pairs[2k+1].  brute != 0 scans all pairs; otherwise uses the cell list.
 * Returns the pair count (pairs may be NULL to count). */
int64_t orc_contact_pairs(const orc_problem *P, const double *u, const uint8_t *broken, int brute,
                          int32_t *pairs)
{
    int64_t n = P->n;
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; ++i) p[i] = P->x[i] + u[i];
    orc_grid g;
    int use_grid = !brute;
    if (use_grid) orc_grid_build(&g, n, p, P->Rc);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = orc_contacts_of(P, p, broken, use_grid ? &g : NULL, i, buf, out);
        for (int64_t t = 0; t < k; ++t) {
            if (pairs) { pairs[2 * total] = (int32_t)i; pairs[2 * total + 1] = (int32_t)out[t]; }
            ++total;
        }
    }
    if (use_grid) orc_grid_free(&g);
    free(p); free(buf); free(out);
    return total;
}

/* A shared-region term of step 5 of orc_forces: the walls idx[0..m-1] at
 * distances dist[] cut W; the term's force density (sign applied) is added to
 * f and its components along each wall's normal go to that wall's reaction. */
static void orc_overlap_term(const orc_problem *P, int m, const int *idx, const double *dist, double sign, double vol,
                             double *f, double *react)
{
    double cut[4];
    orc_ball_cut(P->Rc, dist[0], dist[1], m == 3 ? dist[2] : -P->Rc, cut);
    double V = cut[0];
    if (!(V > 0.0)) return;
    double cbar[3] = {cut[1] / V, cut[2] / V, m == 3 ? cut[3] / V : 0.0}; /* along -n of each wall */
    double rb = sqrt(sq3(cbar[0], cbar[1], cbar[2]));
    if (!(rb > 0.0)) return;
    /* F = -K_n (R_c - rb) V (c - p) / rb with c - p = -sum_k cbar[k] n_k */
    double g = sign * P->Kn * (P->Rc - rb) * V / rb;
    for (int k = 0; k < m; ++k) {
        const double *nk = P->walls + 9 * idx[k];
        for (int a = 0; a < 3; ++a) {
            double fa = g * cbar[k] * nk[a];
            f[a] += fa;
            react[3 * idx[k] + a] -= fa * vol;
        }
    }
}

/* step 5 of orc_forces for the node at p */
static int orc_wall_overlap(const orc_problem *P, const double *p, const double *wall_pos, double vol, double *f,
                            double *react)
{
    int touch[6], nt = 0;
    double dist[6];
    for (int l = 0; l < P->nw && l < 6; ++l) {
        const double *nl = P->walls + 9 * l;
        const double *wl = wall_pos + 3 * l;
        double d = ((p[0] - wl[0]) * nl[0] + (p[1] - wl[1]) * nl[1]) + (p[2] - wl[2]) * nl[2];
        if (d < P->Rc && d > -P->Rc) { touch[nt] = l; dist[nt] = d; ++nt; }
    }
    for (int s = 0; s < nt; ++s)
        for (int t = s + 1; t < nt; ++t) {
            const double *ns = P->walls + 9 * touch[s], *nu = P->walls + 9 * touch[t];
            if (fabs(ns[0] * nu[0] + ns[1] * nu[1] + ns[2] * nu[2]) > 1e-9) continue;
            int idx[2] = {touch[s], touch[t]};
            double dd[2] = {dist[s], dist[t]};
            orc_overlap_term(P, 2, idx, dd, -1.0, vol, f, react);
            for (int r = t + 1; r < nt; ++r) {
                const double *nr = P->walls + 9 * touch[r];
                if (fabs(ns[0] * nr[0] + ns[1] * nr[1] + ns[2] * nr[2]) > 1e-9) continue;
                if (fabs(nu[0] * nr[0] + nu[1] * nr[1] + nu[2] * nr[2]) > 1e-9) continue;
                int id3[3] = {touch[s], touch[t], touch[r]};
                double d3[3] = {dist[s], dist[t], dist[r]};
                orc_overlap_term(P, 3, id3, d3, 1.0, vol, f, react);
            }
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Force density at displacement u (Eq. motion: F_int + F_ext without b).    */
/* ------------------------------------------------------------------------- */
/*
 * For every node i, in this order:
 * 1. Bonds (Eq. peri-damage, Eq. peri2, stretch of Sec. 3.1): for each slot
 *    (i, j) with gamma = 1, xi = x_j - x_i, eta = u_j - u_i,
 *    s = (|xi + eta| - |xi|) / |xi|.  If s > s0 (break_mode 0) or |s| > s0
 *    (break_mode 1) the bond memory becomes 0 (broken[k] = 1) and the bond
 *    carries no force from this evaluation on.  Otherwise
 *    F_i += c s (xi + eta) / |xi + eta| V_j.
 *    Reading: the gamma definition breaks on tension (s > s0); the sentence
 *    before the table says |s| > |s0|; break_mode selects.
 * 2. Contact (Sec. 3.2 and the self-contact section), for each partner j
 *    returned by orc_contacts_of, with d = p_j - p_i and e = d / |d|:
 *    - j in another grain, or same grain with |x_j - x_i| >= R_c:
 *        F_i += -K_n (R_c - |d|) e V_j
 *    - same grain and |x_j - x_i| < R_c (a once-bonded pair):
 *        F_i += c min(0, (|d| - |xi|) / |xi|) e V_j
 *    Reading: |d| = 0 has no direction and contributes nothing.
 *    Normal damping (Sec. 3.3, Eq. damping-force), when v is given and
 *    beta_d != 0, on the same pairs: F_i += beta_d ((v_j - v_i) . e) e V_j.
 *    Reading: the printed law -beta_d (v/|v| . e) e with v = v_j - v_i pushes
 *    approaching points towards each other, while the text says the force acts
 *    against e for them; and its unit-length v gives a force of magnitude
 *    beta_d cos(angle) at any speed, while the text calls the law linear and a
 *    viscoelastic spring.  The dissipative linear law is used.
 * 3. Walls (Sec. 4.1), for each wall l with inward unit normal n_l and current
 *    point w_l: d = (p_i - w_l) . n_l.  If d < R_c the ball of radius R_c
 *    around p_i overlaps the wall in a spherical cap of volume
 *    |S| = (pi/3)(R_c - d)^2 (2 R_c + d) whose centroid lies at
 *    zbar = (pi/4)(R_c^2 - d^2)^2 / |S| from p_i.  Then
 *    F_i += K_n (R_c - zbar) |S| n_l and the wall receives -F V_i.
 *    Reading: the printed volume has (2 R_c - d); that is not the volume of
 *    the cap and makes the force attractive near d = R_c; the printed
 *    centroid formula is only consistent with (2 R_c + d).  d <= -R_c (a node
 *    a whole radius behind the wall) is undefined and flagged ORC_ERR_WALL.
 *    Damping at the wall (Sec. 4.1: e -> e_l, V_y -> |S|, p_y -> c_l, the cap
 *    moving with the wall velocity v_w): F_i += beta_d ((v_w - v_i) . n_l) n_l |S|,
 *    which the wall's reaction includes.
 * 4. Stick-slip friction (Sec. 3.3, Eq. regularized-friction), when v is given
 *    and mu != 0.  For a contact pair with e = d / |d| and the relative velocity
 *    of i with respect to j, v_r = v_i - v_j, the tangential part is
 *    v_t = v_r - (v_r . e) e.  With f_r the magnitude of the pair's repulsion of
 *    step 2 (per volume squared):
 *      F_i += -min(rho |v_t| / (dt (V_i + V_j)), mu f_r) V_j v_t / |v_t|.
 *    Readings: the law acts against the slip of i relative to j, as the text
 *    says (the printed e_perp(y, x) would push along it).  The printed stick
 *    branch (1/eps_f)|v_t| = rho |v_t| / dt is a force density, not a density
 *    per volume squared like f_r; dividing it by V_i + V_j keeps the pair law
 *    antisymmetric (momentum is conserved) and stops the relative tangential
 *    motion of an isolated pair in exactly one step, the property the paper
 *    gives for eps_f = dt / rho.  The stick and slip branches then meet where
 *    |v_t| = v_thr, so the law is min() of the two.  dt = 0 is the Coulomb
 *    limit (v_thr -> 0, slip whenever |v_t| > 0).
 *    At a wall (Sec. 4.1 substitution, the wall rigid): v_r = v_i - v_w,
 *    v_t = v_r - (v_r . n_l) n_l, f_r |S| = K_n (R_c - zbar) |S|, and the stick
 *    branch is the force density that stops v_t in one step:
 *      F_i += -min(rho |v_t| / dt, mu K_n (R_c - zbar) |S|) v_t / |v_t|,
 *    which the wall's reaction includes.
 * 5. Several walls (Sec. 4.1.1), when wall_overlap is set: for every pair of
 *    walls with orthogonal normals that both touch the node, the shared region
 *    W(d_l, d_m, -R_c) of orc_ball_cut (X along -n_l, Y along -n_m) of volume
 *    |S_lm| and centroid c_lm - p_i = -(Mx n_l + My n_m) / |S_lm| contributes
 *    -F_lm with F_lm = -K_n (R_c - |c_lm - p_i|) |S_lm| (c_lm - p_i) / |c_lm - p_i|,
 *    and every triple of mutually orthogonal touching walls contributes +F_lmk
 *    of W(d_l, d_m, d_k), the same form.  Readings: the paper states the
 *    principle without the regions' volumes and centroids, which are computed
 *    here; its triple term carries a stray factor V_x, dropped so that all
 *    terms have the single-wall form; walls that are not orthogonal keep the
 *    plain sum; damping and friction stay single-wall sums (the shared region
 *    has no single wall velocity); the component of a shared-region term along
 *    n_l is the part wall l's reaction takes.
 * With P->frozen set, step 1 keeps the given bond memory (Eq. peri-damage with
 * gamma prescribed) so that two evaluations can be compared on one bond set.
 * Returns error bits.  react (nw*3) receives the total force on each wall.
 */
int orc_forces(const orc_problem *P, const double *u, const double *v, const double *wall_pos, uint8_t *broken,
               double *F, double *react)
{
    const int damp = v != NULL && P->beta_d != 0.0;
    const int fric = v != NULL && P->mu != 0.0;
    int64_t n = P->n;
    int err = 0;
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t *buf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < 3 * n; ++i) p[i] = P->x[i] + u[i];
    for (int l = 0; l < 3 * P->nw; ++l) react[l] = 0.0;

    /* 1. bonds for all rows (each row decides its own slots; a bond's two
     *    directions see negated xi, eta and therefore decide identically).  Rows
     *    write only their own F and slots, so the OpenMP build (for timing on all
     *    host cores) gives the same bits as the serial one. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) {
            if (broken[k]) continue;
            int64_t j = P->col[k];
            double xi[3], eta[3], y[3];
            for (int a = 0; a < 3; ++a) {
                xi[a] = P->x[3 * j + a] - P->x[3 * i + a];
                eta[a] = u[3 * j + a] - u[3 * i + a];
                y[a] = xi[a] + eta[a];
            }
            double L = sqrt(sq3(xi[0], xi[1], xi[2]));
            double l = sqrt(sq3(y[0], y[1], y[2]));
            double s = (l - L) / L;
            int brk = P->break_mode ? (fabs(s) > P->s0) : (s > P->s0);
            if (brk && !P->frozen) { broken[k] = 1; continue; }
            double g = orc_cw(P, L) * s * P->vol[j] / l;
            for (int a = 0; a < 3; ++a) f[a] += g * y[a];
        }
        for (int a = 0; a < 3; ++a) F[3 * i + a] = f[a];
    }

    /* 2. contact, after every row has updated its bond memory (rows again write
     *    only their own F; each thread has its own scratch lists) */
    if (P->contact) {
        orc_grid g;
        orc_grid_build(&g, n, p, P->Rc);
#ifdef _OPENMP
#pragma omp parallel
#endif
        {
        int64_t *tbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        int64_t *tnb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t i = 0; i < n; ++i) {
            int64_t m = orc_contacts_of(P, p, broken, &g, i, tbuf, tnb);
            for (int64_t t = 0; t < m; ++t) {
                int64_t j = tnb[t];
                double d[3], xi[3];
                for (int a = 0; a < 3; ++a) {
                    d[a] = p[3 * j + a] - p[3 * i + a];
                    xi[a] = P->x[3 * j + a] - P->x[3 * i + a];
                }
                double dn = sqrt(sq3(d[0], d[1], d[2]));
                if (dn == 0.0) continue;
                double L = sqrt(sq3(xi[0], xi[1], xi[2]));
                double mag;
                if (P->grain[i] != P->grain[j] || L >= P->Rc) {
                    mag = -P->Kn * (P->Rc - dn);
                } else {
                    double sr = (dn - L) / L;
                    mag = orc_cw(P, L) * (sr < 0.0 ? sr : 0.0);
                }
                for (int a = 0; a < 3; ++a) F[3 * i + a] += mag * (d[a] / dn) * P->vol[j];
                if (damp) {
                    /* Eq. (damping-force), read as the linear dissipative law
                     * beta_d ((v_j - v_i) . e) e with e = d / |d| */
                    double e[3], w = 0.0;
                    for (int a = 0; a < 3; ++a) e[a] = d[a] / dn;
                    for (int a = 0; a < 3; ++a) w += (v[3 * j + a] - v[3 * i + a]) * e[a];
                    for (int a = 0; a < 3; ++a) F[3 * i + a] += P->beta_d * w * e[a] * P->vol[j];
                }
                if (fric) {
                    double e[3], vr[3], vt[3], vn = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        e[a] = d[a] / dn;
                        vr[a] = v[3 * i + a] - v[3 * j + a];
                        vn += vr[a] * e[a];
                    }
                    for (int a = 0; a < 3; ++a) vt[a] = vr[a] - vn * e[a];
                    double vtn = sqrt(sq3(vt[0], vt[1], vt[2]));
                    if (vtn > 0.0) {
                        double slip = P->mu * fabs(mag);
                        double stick = P->dt_f > 0.0 ? P->rho * vtn / (P->dt_f * (P->vol[i] + P->vol[j])) : INFINITY;
                        double f = stick < slip ? stick : slip;
                        for (int a = 0; a < 3; ++a) F[3 * i + a] -= f * (vt[a] / vtn) * P->vol[j];
                    }
                }
            }
        }
        free(tbuf); free(tnb);
        }
        orc_grid_free(&g);
    }

    /* 3. walls (serial: the wall reactions are summed in caller order) */
    for (int64_t i = 0; i < n; ++i) {
        for (int l = 0; l < P->nw; ++l) {
            const double *nl = P->walls + 9 * l;
            const double *wl = wall_pos + 3 * l;
            double d = ((p[3 * i] - wl[0]) * nl[0] + (p[3 * i + 1] - wl[1]) * nl[1]) +
                       (p[3 * i + 2] - wl[2]) * nl[2];
            if (!(d < P->Rc)) continue;
            if (d <= -P->Rc) { err |= ORC_ERR_WALL; continue; }
            double hc = P->Rc - d;
            double Vcap = (ORC_PI / 3.0) * hc * hc * (2.0 * P->Rc + d);
            double q = P->Rc * P->Rc - d * d;
            double zbar = (ORC_PI / 4.0) * q * q / Vcap;
            double mag = P->Kn * (P->Rc - zbar) * Vcap;
            if (damp) {
                /* the wall's points in the cap move with the wall: the pair law
                 * with e = -n, V_y = |S_l| (Sec. 4.1); ((v_w - v_i) . e) e is the
                 * same along n */
                double w = 0.0;
                for (int a = 0; a < 3; ++a) w += (P->walls[9 * l + 6 + a] - v[3 * i + a]) * nl[a];
                mag += P->beta_d * w * Vcap;
            }
            for (int a = 0; a < 3; ++a) {
                F[3 * i + a] += mag * nl[a];
                react[3 * l + a] -= mag * nl[a] * P->vol[i];
            }
            if (fric) {
                double vr[3], vt[3], vn = 0.0;
                for (int a = 0; a < 3; ++a) {
                    vr[a] = v[3 * i + a] - P->walls[9 * l + 6 + a];
                    vn += vr[a] * nl[a];
                }
                for (int a = 0; a < 3; ++a) vt[a] = vr[a] - vn * nl[a];
                double vtn = sqrt(sq3(vt[0], vt[1], vt[2]));
                if (vtn > 0.0) {
                    double slip = P->mu * P->Kn * (P->Rc - zbar) * Vcap;
                    double stick = P->dt_f > 0.0 ? P->rho * vtn / P->dt_f : INFINITY;
                    double f = stick < slip ? stick : slip;
                    for (int a = 0; a < 3; ++a) {
                        F[3 * i + a] -= f * vt[a] / vtn;
                        react[3 * l + a] += f * vt[a] / vtn * P->vol[i];
                    }
                }
            }
        }
        if (P->wall_overlap) err |= orc_wall_overlap(P, p + 3 * i, wall_pos, P->vol[i], F + 3 * i, react);
        for (int a = 0; a < 3; ++a)
            if (!isfinite(F[3 * i + a])) err |= ORC_ERR_NONFINITE;
    }
    free(p); free(buf); free(nb);
    return err;
}

/*
 * Velocity-Verlet (Sec. 5.2) for Eq. (motion): rho u'' = F(u) + b.
 * On entry acc holds a(t) = (F(u(t)) + b) / rho.  Each step:
 *   v <- v + (dt/2) a;  u <- u + dt v;  walls advance w <- w + dt v_wall;
 *   a <- (F(u) + b) / rho;  v <- v + (dt/2) a.
 * Returns the OR of the force error bits; react holds the wall forces of the
 * last evaluation.  impulse (nw*3, nullable) accumulates dt * react after every
 * step's force evaluation: the wall impulse over the steps, rectangle rule on
 * the evaluations at the ends of the steps.
 */
int orc_step(const orc_problem *P, double *u, double *v, double *acc, uint8_t *broken,
             double *wall_pos, double dt, int64_t nsteps, double *F, double *react, double *impulse)
{
    int64_t n = P->n;
    int err = 0;
    double hdt = 0.5 * dt;
    for (int64_t s = 0; s < nsteps; ++s) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < 3 * n; ++i) {
            v[i] = v[i] + hdt * acc[i];
            u[i] = u[i] + dt * v[i];
        }
        for (int l = 0; l < P->nw; ++l)
            for (int a = 0; a < 3; ++a)
                wall_pos[3 * l + a] = wall_pos[3 * l + a] + dt * P->walls[9 * l + 6 + a];
        /* velocity-dependent forces see the half-step velocity v(t + dt/2);
         * the friction's stick branch sees this step's dt */
        orc_problem Q = *P;
        Q.dt_f = dt;
        err |= orc_forces(&Q, u, v, wall_pos, broken, F, react);
        if (impulse)
            for (int l = 0; l < 3 * P->nw; ++l) impulse[l] += dt * react[l];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                acc[3 * i + a] = (F[3 * i + a] + P->b[a]) / P->rho;
                v[3 * i + a] = v[3 * i + a] + hdt * acc[3 * i + a];
            }
    }
    return err;
}

/*
 * Critical time step.  Reading (the paper gives only "stability analysis"):
 * the Silling-Askari bound for explicit PMB integration,
 *   dt_crit = min_i sqrt(2 rho / sum_{j in bonds of i} V_j c / |x_j - x_i|),
 * over nodes with at least one bond, on the initial bond list.
 */
double orc_stable_dt(const orc_problem *P)
{
    double best = INFINITY;
    for (int64_t i = 0; i < P->n; ++i) {
        if (P->rowptr[i + 1] == P->rowptr[i]) continue;
        double sum = 0.0;
        for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) {
            int64_t j = P->col[k];
            double L = sqrt(sq3(P->x[3 * j] - P->x[3 * i], P->x[3 * j + 1] - P->x[3 * i + 1],
                                P->x[3 * j + 2] - P->x[3 * i + 2]));
            sum += P->vol[j] * orc_cw(P, L) / L;
        }
        double dt = sqrt(2.0 * P->rho / sum);
        if (dt < best) best = dt;
    }
    return best;
}

/*
 * Damage (Sec. 3.1.1): phi_i = 1 - (intact bonds of i) / (bonds of i at t = 0),
 * 0 for a node without bonds.  Reading: the sentence in the paper calls the
 * ratio of intact to initial bonds "damage"; that ratio is 1 - phi (it is 1 for
 * an undamaged node), so phi is taken as its complement, counted (not
 * volume-weighted).
 */
void orc_damage(int64_t n, const int64_t *rowptr, const uint8_t *broken, double *phi)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t nb0 = rowptr[i + 1] - rowptr[i], intact = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) intact += broken[k] ? 0 : 1;
        phi[i] = nb0 ? 1.0 - (double)intact / (double)nb0 : 0.0;
    }
}

/*
 * Fragments (split-off pieces; the paper identifies them but gives no
 * algorithm).  Reading: the connected components of the graph whose vertices
 * are the nodes and whose edges are the intact bonds; a fragment is labelled by
 * the smallest node index it contains.  Plain union-find: every intact slot
 * (i, j) joins the sets of i and j (the set's representative is always its
 * smallest member).  label (n) receives each node's fragment label; returns the
 * number of fragments.
 */
static int64_t orc_find(int64_t *parent, int64_t x)
{
    while (parent[x] != x) x = parent[x];
    return x;
}

int64_t orc_fragments(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *broken, int32_t *label)
{
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (broken[k]) continue;
            int64_t a = orc_find(parent, i), b = orc_find(parent, col[k]);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;
        }
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = orc_find(parent, i);
        label[i] = (int32_t)r;
        if (r == i) ++count;
    }
    free(parent);
    return count;
}

/*
 * Per-fragment statistics, fragments in increasing label order: node count,
 * volume, and damage read as the broken fraction of the fragment's initial bond
 * slots, 1 - sum intact / sum initial (0 for a fragment without bonds).
 */
void orc_fragment_stats(int64_t n, const int64_t *rowptr, const uint8_t *broken, const double *vol,
                        const int32_t *label, int64_t nfrag, int64_t *size, double *volume, double *damage)
{
    int64_t *index = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *intact = (int64_t *)calloc((size_t)(nfrag > 0 ? nfrag : 1), sizeof(int64_t));
    int64_t *slots = (int64_t *)calloc((size_t)(nfrag > 0 ? nfrag : 1), sizeof(int64_t));
    int64_t f = 0;
    for (int64_t i = 0; i < n; ++i) index[i] = (label[i] == i) ? f++ : -1;
    for (int64_t q = 0; q < nfrag; ++q) { size[q] = 0; volume[q] = 0.0; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t q = index[label[i]];
        size[q] += 1;
        volume[q] += vol[i];
        slots[q] += rowptr[i + 1] - rowptr[i];
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) intact[q] += broken[k] ? 0 : 1;
    }
    for (int64_t q = 0; q < nfrag; ++q) damage[q] = slots[q] ? 1.0 - (double)intact[q] / (double)slots[q] : 0.0;
    free(index); free(intact); free(slots);
}

/*
 * Total energy for the conservation pin: kinetic sum 1/2 rho V |v|^2, bond
 * energy 1/4 c s^2 |xi| V_i V_j per intact directed bond (the PMB pair
 * potential 1/2 c s^2 |xi| shared by the two directions), and contact spring
 * energy 1/4 K_n (R_c - |d|)^2 V_i V_j per ordered contact pair (spring
 * branch only; the tests that use this keep contacts on the spring branch).
 * Walls are not included.
 */
double orc_energy(const orc_problem *P, const double *u, const double *v, const uint8_t *broken)
{
    int64_t n = P->n;
    double ke = 0.0, pe = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        ke += 0.5 * P->rho * P->vol[i] * sq3(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
        for (int64_t k = P->rowptr[i]; k < P->rowptr[i + 1]; ++k) {
            if (broken[k]) continue;
            int64_t j = P->col[k];
            double xi[3], y[3];
            for (int a = 0; a < 3; ++a) {
                xi[a] = P->x[3 * j + a] - P->x[3 * i + a];
                y[a] = xi[a] + (u[3 * j + a] - u[3 * i + a]);
            }
            double L = sqrt(sq3(xi[0], xi[1], xi[2]));
            double s = (sqrt(sq3(y[0], y[1], y[2])) - L) / L;
            pe += 0.25 * orc_cw(P, L) * s * s * L * P->vol[i] * P->vol[j];
        }
    }
    if (P->contact) {
        int64_t np = orc_contact_pairs(P, u, broken, 0, NULL);
        int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(np > 0 ? np : 1));
        orc_contact_pairs(P, u, broken, 0, pr);
        for (int64_t k = 0; k < np; ++k) {
            int64_t i = pr[2 * k], j = pr[2 * k + 1];
            double dn = sqrt(sq3(P->x[3 * j] + u[3 * j] - P->x[3 * i] - u[3 * i],
                                 P->x[3 * j + 1] + u[3 * j + 1] - P->x[3 * i + 1] - u[3 * i + 1],
                                 P->x[3 * j + 2] + u[3 * j + 2] - P->x[3 * i + 2] - u[3 * i + 2]));
            pe += 0.25 * P->Kn * (P->Rc - dn) * (P->Rc - dn) * P->vol[i] * P->vol[j];
        }
        free(pr);
    }
    return ke + pe;
}
