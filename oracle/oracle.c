/*
 * FP64 CPU oracle for the B-spline x-ray transform (SplineSplat, arXiv 2511.11078).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. The product path
 * (the CUDA library and its Python binding) never calls it and shares no
 * code, header, table or constant with it.
 *
 * Everything is plain, slow, double precision and written from the
 * definitions in the paper:
 *   - Eq. 1: a line {s + t w}, w on the unit sphere.
 *   - Eq. 2: the x-ray transform  Pf(w,s) = integral of f(s + t w) dt.
 *   - Eq. 3: f = sum_k c_k phi(. - k) on the unit lattice (Sec. 2.1), with
 *            phi = beta^n (x) beta^n (x) beta^n a tensor-product B-spline
 *            (Sec. 2.2 uses n = 2; this oracle takes any n in 0..3).
 *   - Eq. 4: Pf(w,s) = sum_k c_k Pphi(w, s - k).  The "contribution" of basis
 *            k is Pphi evaluated at the offset s - k (only its projection on
 *            H_w matters, because Pphi is invariant along w).
 *   - Eq. 5-6: the system matrix [P]_{m,l} = Pphi(w_m, s_m - k_l) used by
 *            least squares; its transpose is the adjoint.
 *   - Algorithm 2 / Algorithm 3: the DDA march with neighbourhood windows
 *            and de-duplication against the two previous steps; the oracle
 *            re-implements it only to check the set of visited bases.
 *
 * Exact footprint (the label generator of Algorithm 1 is replaced by exact
 * quadrature): Pphi(w,p) = int prod_d beta^n(p_d + t w_d) dt.  Each factor is
 * a piecewise polynomial of degree n in t with breaks where p_d + t w_d hits
 * a knot of beta^n.  Between consecutive breaks the product is a polynomial of
 * degree <= 3n, so m-point Gauss-Legendre with 2m - 1 >= 3n is exact up to
 * rounding.
 *
 * Conventions (readings of the paper, stated once here):
 *   - Coefficient k = (kx, ky, kz), 0 <= k < dims, sits at origin + k
 *     (unit lattice), stored C-order c[(kz*ny + ky)*nx + kx].
 *   - beta^0 is the half-open box [-1/2, 1/2) so partition of unity is exact.
 *   - A (ray, basis) pair contributes when the open support cube of the basis
 *     meets the line in a segment of positive length.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXM 16

/* ------------------------------------------------------------------------- */
/* 1-D B-spline (Sec. 2.2; Schoenberg's truncated-power definition)           */
/* ------------------------------------------------------------------------- */

/* beta^n(x) = 1/n! * sum_{k=0}^{n+1} (-1)^k C(n+1,k) (x + (n+1)/2 - k)_+^n.
 * For n >= 1 the function is even, and evaluating at -|x| keeps every
 * surviving term positive-dominated (no cancellation near the right edge). */
double orc_bspline(int n, double x)
{
    if (n == 0) return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    double W = 0.5 * (n + 1);
    double xa = -fabs(x);
    double sum = 0.0, binom = 1.0, fact = 1.0;
    for (int i = 2; i <= n; ++i) fact *= i;
    for (int k = 0; k <= n + 1; ++k) {
        double u = xa + W - k;
        if (u > 0.0) {
            double pw = 1.0;
            for (int i = 0; i < n; ++i) pw *= u;
            sum += ((k & 1) ? -binom : binom) * pw;
        }
        binom = binom * (n + 1 - k) / (k + 1);
    }
    double v = sum / fact;
    return v > 0.0 ? v : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule on [-1, 1] (Newton iteration on P_m, three-term       */
/* recurrence for the Legendre polynomials).                                 */
/* ------------------------------------------------------------------------- */
int orc_gauss_legendre(int m, double *x, double *w)
{
    if (m < 1 || m > ORC_MAXM) return -1;
    for (int i = 0; i < m; ++i) {
        double z = cos(M_PI * (i + 0.75) / (m + 0.5)), pm = 0.0, pm1 = 0.0, dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            /* P_m(z) and P_{m-1}(z) by the three-term recurrence */
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= m; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            pm = p1;
            pm1 = p0;
            dp = m * (z * pm - pm1) / (z * z - 1.0);
            double dz = pm / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= m; ++j) {
            double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = m * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Number of Gauss-Legendre nodes that integrate a degree-3n polynomial
 * exactly: the smallest m with 2m - 1 >= 3n. */
int orc_gl_order(int n) { return (3 * n + 2) / 2 > 0 ? (3 * n + 2) / 2 : 1; }

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------- */
/* Exact footprint Pphi(w, p) (Eq. 2 applied to phi; Eq. 4's contribution)   */
/* ------------------------------------------------------------------------- */
double orc_footprint_m(int n, const double *w, const double *p, int m)
{
    const double W = 0.5 * (n + 1);
    double tlo = -INFINITY, thi = INFINITY, cst = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (w[d] == 0.0) {
            double b = orc_bspline(n, p[d]);
            if (b == 0.0) return 0.0;
            cst *= b;
        } else {
            double t1 = (-W - p[d]) / w[d], t2 = (W - p[d]) / w[d];
            double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
            if (lo > tlo) tlo = lo;
            if (hi < thi) thi = hi;
        }
    }
    if (!(thi > tlo)) return 0.0;
    double br[3 * 8 + 2];
    int nb = 0;
    br[nb++] = tlo;
    for (int d = 0; d < 3; ++d) {
        if (w[d] == 0.0) continue;
        for (int j = 1; j <= n; ++j) {
            double t = (-W + j - p[d]) / w[d];
            if (t > tlo && t < thi) br[nb++] = t;
        }
    }
    br[nb++] = thi;
    qsort(br, nb, sizeof(double), cmp_double);
    double gx[ORC_MAXM], gw[ORC_MAXM];
    orc_gauss_legendre(m, gx, gw);
    double total = 0.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double a = br[i], b = br[i + 1];
        if (!(b > a)) continue;
        double half = 0.5 * (b - a), mid = 0.5 * (a + b), acc = 0.0;
        for (int q = 0; q < m; ++q) {
            double t = mid + half * gx[q], v = 1.0;
            for (int d = 0; d < 3; ++d)
                if (w[d] != 0.0) v *= orc_bspline(n, p[d] + t * w[d]);
            acc += gw[q] * v;
        }
        total += half * acc;
    }
    return total * cst;
}

double orc_footprint(int n, const double *w, const double *p)
{
    return orc_footprint_m(n, w, p, orc_gl_order(n));
}

void orc_footprint_batch(int n, long long count, const double *w, const double *p, double *out)
{
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < count; ++i) out[i] = orc_footprint(n, w + 3 * i, p + 3 * i);
}

/* ------------------------------------------------------------------------- */
/* Geometry (Eq. 1): rays given directly, parallel views, cone views.        */
/* Ray r of a view-based geometry is pixel (iu, iv) of view v with           */
/* r = (v * nv + iv) * nu + iu.  Pixel centre                                */
/*   q = det_center + (iu - (nu-1)/2) det_u + (iv - (nv-1)/2) det_v.         */
/* Parallel: w = dir / |dir|, s = q.  Cone: s = source, w = (q-s)/|q-s|.     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int kind; /* 0 = explicit rays, 1 = parallel views, 2 = cone views */
    int n_views, nu, nv;
    long long n_rays;
    const double *ray_w, *ray_s;                   /* kind 0: [n_rays][3] */
    const double *dir_or_src, *det_c, *det_u, *det_v; /* kinds 1, 2: [n_views][3] */
} orc_geom;

long long orc_geom_rays(const orc_geom *g)
{
    return g->kind == 0 ? g->n_rays : (long long)g->n_views * g->nu * g->nv;
}

int orc_geom_ray(const orc_geom *g, long long r, double *s, double *w)
{
    if (g->kind == 0) {
        double nrm = 0.0;
        for (int d = 0; d < 3; ++d) nrm += g->ray_w[3 * r + d] * g->ray_w[3 * r + d];
        nrm = sqrt(nrm);
        for (int d = 0; d < 3; ++d) { w[d] = g->ray_w[3 * r + d] / nrm; s[d] = g->ray_s[3 * r + d]; }
        return 0;
    }
    long long per = (long long)g->nu * g->nv;
    int v = (int)(r / per);
    long long rem = r - (long long)v * per;
    int iv = (int)(rem / g->nu), iu = (int)(rem - (long long)iv * g->nu);
    double a = iu - 0.5 * (g->nu - 1), b = iv - 0.5 * (g->nv - 1);
    double q[3];
    for (int d = 0; d < 3; ++d)
        q[d] = g->det_c[3 * v + d] + a * g->det_u[3 * v + d] + b * g->det_v[3 * v + d];
    double dir[3];
    if (g->kind == 1) {
        for (int d = 0; d < 3; ++d) { dir[d] = g->dir_or_src[3 * v + d]; s[d] = q[d]; }
    } else {
        for (int d = 0; d < 3; ++d) { dir[d] = q[d] - g->dir_or_src[3 * v + d]; s[d] = g->dir_or_src[3 * v + d]; }
    }
    double nrm = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int d = 0; d < 3; ++d) w[d] = dir[d] / nrm;
    return 0;
}

void orc_geom_all_rays(const orc_geom *g, double *s, double *w)
{
    long long nr = orc_geom_rays(g);
    for (long long r = 0; r < nr; ++r) orc_geom_ray(g, r, s + 3 * r, w + 3 * r);
}

/* ------------------------------------------------------------------------- */
/* Pair enumeration: every k in the grid whose open support cube             */
/* [k - W, k + W]^3 meets the line in a segment of positive length.          */
/* Plain interval geometry, independent of the DDA of Algorithm 2.           */
/* ------------------------------------------------------------------------- */
static int axis_interval(int n, double p, double w, double *lo, double *hi)
{
    const double W = 0.5 * (n + 1);
    if (w == 0.0) {
        if (orc_bspline(n, p) == 0.0) return 0;
        *lo = -INFINITY; *hi = INFINITY;
        return 1;
    }
    double t1 = (-W - p) / w, t2 = (W - p) / w;
    *lo = t1 < t2 ? t1 : t2;
    *hi = t1 < t2 ? t2 : t1;
    return 1;
}

static void index_range(double xlo, double xhi, double W, double org, int nk, int *k0, int *k1)
{
    /* candidate k with |x - org - k| < W for some x in [xlo, xhi], one more
     * on each side: xlo and xhi are rounded, and the interval test of
     * for_each_pair alone must decide which bases count */
    double a = xlo - org - W, b = xhi - org + W;
    double fa = floor(a) - 1.0, fb = ceil(b) + 1.0;
    if (fa < 0) fa = 0;
    if (fa > nk) fa = nk;
    if (fb > nk - 1) fb = nk - 1;
    if (fb < -1) fb = -1;
    *k0 = (int)fa;
    *k1 = (int)fb;
}

typedef void (*orc_pair_fn)(void *ctx, long long kidx, const int *k, const double *p);

static void for_each_pair(int n, const int *dims, const double *org, const double *s,
                          const double *w, orc_pair_fn fn, void *ctx)
{
    const double W = 0.5 * (n + 1);
    for (int kx = 0; kx < dims[0]; ++kx) {
        double px = s[0] - (org[0] + kx), lx, hx;
        if (!axis_interval(n, px, w[0], &lx, &hx)) continue;
        double y0, y1;
        if (w[1] == 0.0) { y0 = y1 = s[1]; }
        else if (isinf(lx) || isinf(hx)) { y0 = -INFINITY; y1 = INFINITY; }
        else { y0 = s[1] + lx * w[1]; y1 = s[1] + hx * w[1]; if (y0 > y1) { double t = y0; y0 = y1; y1 = t; } }
        int ky0, ky1;
        if (isinf(y0) || isinf(y1)) { ky0 = 0; ky1 = dims[1] - 1; }
        else index_range(y0, y1, W, org[1], dims[1], &ky0, &ky1);
        for (int ky = ky0; ky <= ky1; ++ky) {
            double py = s[1] - (org[1] + ky), ly, hy;
            if (!axis_interval(n, py, w[1], &ly, &hy)) continue;
            double lxy = lx > ly ? lx : ly, hxy = hx < hy ? hx : hy;
            if (!(hxy > lxy)) continue;
            double z0, z1;
            if (w[2] == 0.0) { z0 = z1 = s[2]; }
            else if (isinf(lxy) || isinf(hxy)) { z0 = -INFINITY; z1 = INFINITY; }
            else { z0 = s[2] + lxy * w[2]; z1 = s[2] + hxy * w[2]; if (z0 > z1) { double t = z0; z0 = z1; z1 = t; } }
            int kz0, kz1;
            if (isinf(z0) || isinf(z1)) { kz0 = 0; kz1 = dims[2] - 1; }
            else index_range(z0, z1, W, org[2], dims[2], &kz0, &kz1);
            for (int kz = kz0; kz <= kz1; ++kz) {
                double pz = s[2] - (org[2] + kz), lz, hz;
                if (!axis_interval(n, pz, w[2], &lz, &hz)) continue;
                double l3 = lxy > lz ? lxy : lz, h3 = hxy < hz ? hxy : hz;
                if (!(h3 > l3)) continue;
                int k[3] = {kx, ky, kz};
                double p[3] = {px, py, pz};
                long long kidx = ((long long)kz * dims[1] + ky) * dims[0] + kx;
                fn(ctx, kidx, k, p);
            }
        }
    }
}

/* ---------------- forward / adjoint, route A (Eq. 4, Eq. 6) ---------------- */
typedef struct { int n; const double *w; const double *c; double sum; long long count; } fwd_ctx;

static void fwd_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    fwd_ctx *x = (fwd_ctx *)vctx;
    x->sum += x->c[kidx] * orc_footprint(x->n, x->w, p);
    x->count += 1;
}

static void count_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)kidx; (void)k; (void)p;
    ((fwd_ctx *)vctx)->count += 1;
}

void orc_forward(int n, const int *dims, const double *org, const double *c, const orc_geom *g,
                 double *y, int nthreads)
{
    long long nr = orc_geom_rays(g);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
    for (long long r = 0; r < nr; ++r) {
        double s[3], w[3];
        orc_geom_ray(g, r, s, w);
        fwd_ctx x = {n, w, c, 0.0, 0};
        for_each_pair(n, dims, org, s, w, fwd_visit, &x);
        y[r] = x.sum;
    }
}

/* Forward on a subset of rays (indices into the geometry). */
void orc_forward_subset(int n, const int *dims, const double *org, const double *c, const orc_geom *g,
                        long long count, const long long *rays, double *y, long long *pairs, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4)
    for (long long i = 0; i < count; ++i) {
        double s[3], w[3];
        orc_geom_ray(g, rays[i], s, w);
        fwd_ctx x = {n, w, c, 0.0, 0};
        for_each_pair(n, dims, org, s, w, fwd_visit, &x);
        y[i] = x.sum;
        if (pairs) pairs[i] = x.count;
    }
}

long long orc_count_pairs(int n, const int *dims, const double *org, const orc_geom *g, long long *per_ray)
{
    long long nr = orc_geom_rays(g), total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
    for (long long r = 0; r < nr; ++r) {
        double s[3], w[3];
        orc_geom_ray(g, r, s, w);
        fwd_ctx x = {n, w, NULL, 0.0, 0};
        for_each_pair(n, dims, org, s, w, count_visit, &x);
        if (per_ray) per_ray[r] = x.count;
        total += x.count;
    }
    return total;
}

typedef struct { int n; const double *w; double yr; double *c; } adj_ctx;

static void adj_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    adj_ctx *x = (adj_ctx *)vctx;
    x->c[kidx] += x->yr * orc_footprint(x->n, x->w, p);
}

/* Adjoint (transpose of Eq. 6): c_k = sum_r y_r Pphi(w_r, s_r - k).
 * Overwrites c.  Serial scatter over rays: the plain definition. */
void orc_adjoint(int n, const int *dims, const double *org, const double *y, const orc_geom *g, double *c)
{
    long long nk = (long long)dims[0] * dims[1] * dims[2], nr = orc_geom_rays(g);
    memset(c, 0, sizeof(double) * nk);
    for (long long r = 0; r < nr; ++r) {
        if (y[r] == 0.0) continue;
        double s[3], w[3];
        orc_geom_ray(g, r, s, w);
        adj_ctx x = {n, w, y[r], c};
        for_each_pair(n, dims, org, s, w, adj_visit, &x);
    }
}

/* Adjoint restricted to a subset of rays: c_k = sum_{i} y_i Pphi(w_{r_i},
 * s_{r_i} - k) over the listed rays (the rows of Eq. 6 they index); same
 * definition as orc_adjoint, parallel over rays.  Grids of up to 2^24
 * coefficients use one private accumulation buffer per thread; larger ones
 * add into c directly with atomic adds (a private copy of a 512^3 grid per
 * thread would not fit in host memory).  Overwrites c; pairs[0] = pair
 * count. */
static void adj_visit_atomic(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    adj_ctx *x = (adj_ctx *)vctx;
    const double v = x->yr * orc_footprint(x->n, x->w, p);
#pragma omp atomic
    x->c[kidx] += v;
}

void orc_adjoint_subset(int n, const int *dims, const double *org, const double *y, const orc_geom *g,
                        long long count, const long long *rays, double *c, long long *pairs, int nthreads)
{
    long long nk = (long long)dims[0] * dims[1] * dims[2];
    memset(c, 0, sizeof(double) * nk);
    long long np = 0;
    const int shared = nk > (1LL << 24);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel reduction(+ : np)
    {
        double *priv = shared ? c : (double *)calloc(nk, sizeof(double));
        fwd_ctx cnt = {n, NULL, NULL, 0.0, 0};
#pragma omp for schedule(dynamic, 4)
        for (long long i = 0; i < count; ++i) {
            double s[3], w[3];
            orc_geom_ray(g, rays[i], s, w);
            adj_ctx x = {n, w, y[i], priv};
            for_each_pair(n, dims, org, s, w, shared ? adj_visit_atomic : adj_visit, &x);
            cnt.w = w;
            for_each_pair(n, dims, org, s, w, count_visit, &cnt);
        }
        np += cnt.count;
        if (!shared) {
#pragma omp critical
            for (long long k = 0; k < nk; ++k) c[k] += priv[k];
            free(priv);
        }
    }
    if (pairs) pairs[0] = np;
}

/* Adjoint at selected coefficients: c_k = sum over every ray of the geometry
 * whose line meets the support cube of k.  Used for sampled checks at sizes
 * where the full scatter is too slow. */
void orc_adjoint_at(int n, const int *dims, const double *org, const double *y, const orc_geom *g,
                    long long count, const long long *kidx, double *out, long long *pairs, int nthreads)
{
    long long nr = orc_geom_rays(g);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (long long i = 0; i < count; ++i) {
        long long kk = kidx[i];
        int kx = (int)(kk % dims[0]), ky = (int)((kk / dims[0]) % dims[1]), kz = (int)(kk / ((long long)dims[0] * dims[1]));
        double ctr[3] = {org[0] + kx, org[1] + ky, org[2] + kz};
        double sum = 0.0;
        long long np = 0;
#pragma omp parallel for schedule(static) reduction(+ : sum, np)
        for (long long r = 0; r < nr; ++r) {
            double s[3], w[3], p[3], lo = -INFINITY, hi = INFINITY;
            orc_geom_ray(g, r, s, w);
            int ok = 1;
            for (int d = 0; d < 3 && ok; ++d) {
                double a, b;
                p[d] = s[d] - ctr[d];
                if (!axis_interval(n, p[d], w[d], &a, &b)) { ok = 0; break; }
                if (a > lo) lo = a;
                if (b < hi) hi = b;
            }
            if (!ok || !(hi > lo)) continue;
            sum += y[r] * orc_footprint(n, w, p);
            np += 1;
        }
        out[i] = sum;
        if (pairs) pairs[i] = np;
    }
}

/* Adjoint at selected coefficients of a view geometry, visiting for each
 * coefficient and view only the detector pixels whose ray can meet the
 * coefficient's support cube: the pixel bounding box (one pixel of margin)
 * of the 8 cube corners projected onto the detector plane along the view's
 * direction (parallel) or through its source (cone).  The support is
 * convex, so every ray that meets it passes through the hull of the
 * projected corners; a corner at or behind the source plane keeps the whole
 * detector.  Each candidate ray then gets the same exact pair test and
 * footprint as orc_adjoint_at, so the result is the same sum (for full-size
 * sampled checks where looping over every ray per coefficient is too slow).
 */
static int view_pixel_window(const orc_geom *g, int v, const double *lo, const double *hi, int *u0, int *u1,
                             int *v0, int *v1)
{
    const double *dc = g->det_c + 3 * v, *du = g->det_u + 3 * v, *dv = g->det_v + 3 * v;
    const double *src = g->dir_or_src + 3 * v;
    double nrm[3] = {du[1] * dv[2] - du[2] * dv[1], du[2] * dv[0] - du[0] * dv[2], du[0] * dv[1] - du[1] * dv[0]};
    /* (a, b) of a point P on the plane: solve the 2x2 normal equations of
       P - dc = a du + b dv */
    const double guu = du[0] * du[0] + du[1] * du[1] + du[2] * du[2];
    const double gvv = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2];
    const double guv = du[0] * dv[0] + du[1] * dv[1] + du[2] * dv[2];
    const double det = guu * gvv - guv * guv;
    if (!(det > 0.0)) return 0;
    double amin = INFINITY, amax = -INFINITY, bmin = INFINITY, bmax = -INFINITY;
    for (int corner = 0; corner < 8; ++corner) {
        const double x[3] = {(corner & 1) ? hi[0] : lo[0], (corner & 2) ? hi[1] : lo[1], (corner & 4) ? hi[2] : lo[2]};
        double P[3];
        if (g->kind == 1) {
            const double den = src[0] * nrm[0] + src[1] * nrm[1] + src[2] * nrm[2];
            if (den == 0.0) return 0;
            const double t = ((x[0] - dc[0]) * nrm[0] + (x[1] - dc[1]) * nrm[1] + (x[2] - dc[2]) * nrm[2]) / den;
            for (int d = 0; d < 3; ++d) P[d] = x[d] - t * src[d];
        } else {
            const double num = (dc[0] - src[0]) * nrm[0] + (dc[1] - src[1]) * nrm[1] + (dc[2] - src[2]) * nrm[2];
            const double den = (x[0] - src[0]) * nrm[0] + (x[1] - src[1]) * nrm[1] + (x[2] - src[2]) * nrm[2];
            if (!(num * den > 0.0)) return 0; /* corner on or behind the source plane */
            const double lam = num / den;
            for (int d = 0; d < 3; ++d) P[d] = src[d] + lam * (x[d] - src[d]);
        }
        const double r[3] = {P[0] - dc[0], P[1] - dc[1], P[2] - dc[2]};
        const double ru = r[0] * du[0] + r[1] * du[1] + r[2] * du[2];
        const double rv = r[0] * dv[0] + r[1] * dv[1] + r[2] * dv[2];
        const double a = (gvv * ru - guv * rv) / det, b = (guu * rv - guv * ru) / det;
        if (a < amin) amin = a;
        if (a > amax) amax = a;
        if (b < bmin) bmin = b;
        if (b > bmax) bmax = b;
    }
    const double cu = 0.5 * (g->nu - 1), cv = 0.5 * (g->nv - 1);
    double fu0 = floor(amin + cu) - 1.0, fu1 = ceil(amax + cu) + 1.0;
    double fv0 = floor(bmin + cv) - 1.0, fv1 = ceil(bmax + cv) + 1.0;
    if (fu0 < 0.0) fu0 = 0.0;
    if (fv0 < 0.0) fv0 = 0.0;
    if (fu1 > g->nu - 1) fu1 = g->nu - 1;
    if (fv1 > g->nv - 1) fv1 = g->nv - 1;
    *u0 = (int)fu0;
    *u1 = (int)fu1;
    *v0 = (int)fv0;
    *v1 = (int)fv1;
    return 1;
}

void orc_adjoint_at_views(int n, const int *dims, const double *org, const double *y, const orc_geom *g,
                          long long count, const long long *kidx, double *out, long long *pairs, int nthreads)
{
    const double W = 0.5 * (n + 1);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (long long i = 0; i < count; ++i) {
        long long kk = kidx[i];
        int kx = (int)(kk % dims[0]), ky = (int)((kk / dims[0]) % dims[1]), kz = (int)(kk / ((long long)dims[0] * dims[1]));
        double ctr[3] = {org[0] + kx, org[1] + ky, org[2] + kz};
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = ctr[d] - W;
            hi[d] = ctr[d] + W;
        }
        double sum = 0.0;
        long long np = 0;
        for (int v = 0; v < g->n_views; ++v) {
            int u0 = 0, u1 = g->nu - 1, v0 = 0, v1 = g->nv - 1;
            if (!view_pixel_window(g, v, lo, hi, &u0, &u1, &v0, &v1)) {
                u0 = 0;
                u1 = g->nu - 1;
                v0 = 0;
                v1 = g->nv - 1;
            }
            for (int iv = v0; iv <= v1; ++iv)
                for (int iu = u0; iu <= u1; ++iu) {
                    const long long r = ((long long)v * g->nv + iv) * g->nu + iu;
                    double s[3], w[3], p[3], tlo = -INFINITY, thi = INFINITY;
                    orc_geom_ray(g, r, s, w);
                    int ok = 1;
                    for (int d = 0; d < 3 && ok; ++d) {
                        double a, b;
                        p[d] = s[d] - ctr[d];
                        if (!axis_interval(n, p[d], w[d], &a, &b)) { ok = 0; break; }
                        if (a > tlo) tlo = a;
                        if (b < thi) thi = b;
                    }
                    if (!ok || !(thi > tlo)) continue;
                    sum += y[r] * orc_footprint(n, w, p);
                    np += 1;
                }
        }
        out[i] = sum;
        if (pairs) pairs[i] = np;
    }
}

/* ------------------------------------------------------------------------- */
/* Route B: integral of f along the ray, split at every knot plane crossing. */
/* On each piece f(s + t w) is a polynomial of degree <= 3n in t, so m-point */
/* Gauss-Legendre of the direct spline evaluation (Eq. 3) is exact.          */
/* ------------------------------------------------------------------------- */
static double eval_spline(int n, const int *dims, const double *org, const double *c, const double *x)
{
    const double W = 0.5 * (n + 1);
    int lo[3], hi[3];
    double u[3];
    for (int d = 0; d < 3; ++d) {
        u[d] = x[d] - org[d];
        double a = ceil(u[d] - W), b = floor(u[d] + W);
        if (a < 0) a = 0;
        if (b > dims[d] - 1) b = dims[d] - 1;
        lo[d] = (int)a; hi[d] = (int)b;
        if (lo[d] > hi[d]) return 0.0;
    }
    double f = 0.0;
    for (int kz = lo[2]; kz <= hi[2]; ++kz) {
        double bz = orc_bspline(n, u[2] - kz);
        if (bz == 0.0) continue;
        for (int ky = lo[1]; ky <= hi[1]; ++ky) {
            double by = orc_bspline(n, u[1] - ky);
            if (by == 0.0) continue;
            for (int kx = lo[0]; kx <= hi[0]; ++kx) {
                double bx = orc_bspline(n, u[0] - kx);
                f += c[((long long)kz * dims[1] + ky) * dims[0] + kx] * bx * by * bz;
            }
        }
    }
    return f;
}

double orc_eval_spline(int n, const int *dims, const double *org, const double *c, const double *x)
{
    return eval_spline(n, dims, org, c, x);
}

static double ray_integral_segmented(int n, const int *dims, const double *org, const double *c,
                                     const double *s, const double *w)
{
    const double W = 0.5 * (n + 1), kap = W - floor(W);
    double tlo = -INFINITY, thi = INFINITY;
    for (int d = 0; d < 3; ++d) {
        double a = org[d] - W, b = org[d] + dims[d] - 1 + W;
        if (w[d] == 0.0) {
            if (!(s[d] > a && s[d] < b)) return 0.0;
            continue;
        }
        double t1 = (a - s[d]) / w[d], t2 = (b - s[d]) / w[d];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tlo) tlo = lo;
        if (hi < thi) thi = hi;
    }
    if (!(thi > tlo)) return 0.0;
    int cap = 2 + 3 * (dims[0] + dims[1] + dims[2] + 8);
    double *br = (double *)malloc(sizeof(double) * cap);
    int nb = 0;
    br[nb++] = tlo;
    for (int d = 0; d < 3; ++d) {
        if (w[d] == 0.0) continue;
        /* planes x_d = org_d + j + kap - ... : all x with x - org_d - kap in Z */
        double x0 = s[d] + tlo * w[d], x1 = s[d] + thi * w[d];
        if (x0 > x1) { double t = x0; x0 = x1; x1 = t; }
        double j0 = ceil(x0 - org[d] - kap), j1 = floor(x1 - org[d] - kap);
        for (double j = j0; j <= j1 && nb < cap - 1; j += 1.0) {
            double t = (org[d] + kap + j - s[d]) / w[d];
            if (t > tlo && t < thi) br[nb++] = t;
        }
    }
    br[nb++] = thi;
    qsort(br, nb, sizeof(double), cmp_double);
    int m = orc_gl_order(n);
    double gx[ORC_MAXM], gw[ORC_MAXM];
    orc_gauss_legendre(m, gx, gw);
    double total = 0.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double a = br[i], b = br[i + 1];
        if (!(b > a)) continue;
        double half = 0.5 * (b - a), mid = 0.5 * (a + b), acc = 0.0;
        for (int q = 0; q < m; ++q) {
            double t = mid + half * gx[q], x[3];
            for (int d = 0; d < 3; ++d) x[d] = s[d] + t * w[d];
            acc += gw[q] * eval_spline(n, dims, org, c, x);
        }
        total += half * acc;
    }
    free(br);
    return total;
}

void orc_forward_segmented(int n, const int *dims, const double *org, const double *c, const orc_geom *g,
                           long long count, const long long *rays, double *y, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    long long nr = rays ? count : orc_geom_rays(g);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long i = 0; i < nr; ++i) {
        double s[3], w[3];
        orc_geom_ray(g, rays ? rays[i] : i, s, w);
        y[i] = ray_integral_segmented(n, dims, org, c, s, w);
    }
}

/* ------------------------------------------------------------------------- */
/* Classic voxel path lengths (Siddon's method: sort every voxel-face        */
/* crossing, the voxel between two crossings gets the segment length).       */
/* The voxel DDA that degree 0 must reproduce (Sec. 1).                       */
/* ------------------------------------------------------------------------- */
static double siddon_ray(const int *dims, const double *org, const double *c, const double *s, const double *w)
{
    double tlo = -INFINITY, thi = INFINITY;
    for (int d = 0; d < 3; ++d) {
        double a = org[d] - 0.5, b = org[d] + dims[d] - 0.5;
        if (w[d] == 0.0) {
            if (!(s[d] >= a && s[d] < b)) return 0.0;
            continue;
        }
        double t1 = (a - s[d]) / w[d], t2 = (b - s[d]) / w[d];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tlo) tlo = lo;
        if (hi < thi) thi = hi;
    }
    if (!(thi > tlo)) return 0.0;
    int cap = dims[0] + dims[1] + dims[2] + 8;
    double *br = (double *)malloc(sizeof(double) * cap);
    int nb = 0;
    br[nb++] = tlo;
    for (int d = 0; d < 3; ++d) {
        if (w[d] == 0.0) continue;
        for (int j = 0; j < dims[d] - 1; ++j) {
            double t = (org[d] + j + 0.5 - s[d]) / w[d];
            if (t > tlo && t < thi) br[nb++] = t;
        }
    }
    br[nb++] = thi;
    qsort(br, nb, sizeof(double), cmp_double);
    double total = 0.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double len = br[i + 1] - br[i];
        if (!(len > 0)) continue;
        double tm = 0.5 * (br[i] + br[i + 1]);
        int k[3], ok = 1;
        for (int d = 0; d < 3; ++d) {
            k[d] = (int)floor(s[d] + tm * w[d] - org[d] + 0.5);
            if (k[d] < 0 || k[d] >= dims[d]) ok = 0;
        }
        if (ok) total += len * c[((long long)k[2] * dims[1] + k[1]) * dims[0] + k[0]];
    }
    free(br);
    return total;
}

void orc_siddon(const int *dims, const double *org, const double *c, const orc_geom *g, double *y)
{
    long long nr = orc_geom_rays(g);
#pragma omp parallel for schedule(dynamic, 16)
    for (long long r = 0; r < nr; ++r) {
        double s[3], w[3];
        orc_geom_ray(g, r, s, w);
        y[r] = siddon_ray(dims, org, c, s, w);
    }
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 + Algorithm 3 re-implemented (FP64) to check the enumeration:  */
/* Amanatides-Woo voxel traversal of the box dilated by R cells; at each     */
/* crossed cell k the window {l : l_d* = k_d*, |l - k|_inf <= R} minus the   */
/* windows kept from the two previous steps.  Emits linear indices of l in   */
/* the grid (bases outside the grid have zero coefficient).                  */
/* Returns the number of emitted bases (-1 if out_cap is too small);         */
/* *max_cells_per_slab gets the largest number of consecutive cells that     */
/* share the dominant-axis index (Sec. 2.1, second observation).             */
/* ------------------------------------------------------------------------- */
typedef struct { int k[3]; } cell3;

long long orc_dda_visit(int n, int R, const int *dims, const double *org, const double *s_in, const double *w,
                        long long *out, long long out_cap, int *max_cells_per_slab, long long *n_cells)
{
    (void)n;
    double s[3];
    for (int d = 0; d < 3; ++d) s[d] = s_in[d] - org[d]; /* index coordinates */
    int dstar = 0;
    for (int d = 1; d < 3; ++d) if (fabs(w[d]) > fabs(w[dstar])) dstar = d;
    /* ray against the dilated box [-1/2 - R, N - 1/2 + R] */
    double tlo = -INFINITY, thi = INFINITY;
    for (int d = 0; d < 3; ++d) {
        double a = -0.5 - R, b = dims[d] - 0.5 + R;
        if (w[d] == 0.0) {
            if (!(s[d] >= a && s[d] < b)) { *max_cells_per_slab = 0; *n_cells = 0; return 0; }
            continue;
        }
        double t1 = (a - s[d]) / w[d], t2 = (b - s[d]) / w[d];
        double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
        if (lo > tlo) tlo = lo;
        if (hi < thi) thi = hi;
    }
    *max_cells_per_slab = 0;
    *n_cells = 0;
    if (!(thi > tlo)) return 0;
    /* first crossed cell: the cell holding the entry point (nudged inside) */
    int k[3], step[3];
    double tmax[3], tdel[3];
    double tin = tlo + 1e-9 * (thi - tlo);
    for (int d = 0; d < 3; ++d) {
        double x = s[d] + tin * w[d];
        k[d] = (int)floor(x + 0.5);
        if (k[d] < -R) k[d] = -R;
        if (k[d] > dims[d] - 1 + R) k[d] = dims[d] - 1 + R;
        if (w[d] > 0) { step[d] = 1; tmax[d] = (k[d] + 0.5 - s[d]) / w[d]; tdel[d] = 1.0 / w[d]; }
        else if (w[d] < 0) { step[d] = -1; tmax[d] = (k[d] - 0.5 - s[d]) / w[d]; tdel[d] = -1.0 / w[d]; }
        else { step[d] = 0; tmax[d] = INFINITY; tdel[d] = INFINITY; }
    }
    int span = 2 * R + 1, wsz = span * span * span;
    cell3 *hist1 = (cell3 *)malloc(sizeof(cell3) * wsz), *hist2 = (cell3 *)malloc(sizeof(cell3) * wsz);
    cell3 *cur = (cell3 *)malloc(sizeof(cell3) * wsz);
    int n1 = 0, n2 = 0;
    long long emitted = 0;
    int run = 0, last_slab = -(1 << 30);
    int ok_cap = 1;
    for (;;) {
        int inside = 1;
        for (int d = 0; d < 3; ++d) if (k[d] < -R || k[d] > dims[d] - 1 + R) inside = 0;
        if (!inside) break;
        *n_cells += 1;
        if (k[dstar] == last_slab) run += 1; else { run = 1; last_slab = k[dstar]; }
        if (run > *max_cells_per_slab) *max_cells_per_slab = run;
        /* Algorithm 3: the window minus the two previous (de-duplicated) sets */
        int nc = 0;
        int l[3];
        int a0 = dstar == 0 ? 1 : 0, b0 = dstar == 2 ? 1 : 2;
        for (int da = -R; da <= R; ++da)
            for (int db = -R; db <= R; ++db) {
                l[dstar] = k[dstar];
                l[a0] = k[a0] + da;
                l[b0] = k[b0] + db;
                int dup = 0;
                for (int i = 0; i < n1 && !dup; ++i)
                    if (hist1[i].k[0] == l[0] && hist1[i].k[1] == l[1] && hist1[i].k[2] == l[2]) dup = 1;
                for (int i = 0; i < n2 && !dup; ++i)
                    if (hist2[i].k[0] == l[0] && hist2[i].k[1] == l[1] && hist2[i].k[2] == l[2]) dup = 1;
                if (dup) continue;
                cur[nc].k[0] = l[0]; cur[nc].k[1] = l[1]; cur[nc].k[2] = l[2];
                nc++;
                if (l[0] >= 0 && l[0] < dims[0] && l[1] >= 0 && l[1] < dims[1] && l[2] >= 0 && l[2] < dims[2]) {
                    if (emitted < out_cap) out[emitted] = ((long long)l[2] * dims[1] + l[1]) * dims[0] + l[0];
                    else ok_cap = 0;
                    emitted++;
                }
            }
        /* (N^-2, N^-1) <- (N^-1, N) */
        cell3 *tmp = hist2; hist2 = hist1; n2 = n1; hist1 = cur; n1 = nc; cur = tmp;
        /* DDA_Step: advance along the axis whose next face is nearest
         * (ties: lowest axis index) */
        int ax = 0;
        for (int d = 1; d < 3; ++d) if (tmax[d] < tmax[ax]) ax = d;
        if (!(tmax[ax] < thi)) break;
        k[ax] += step[ax];
        tmax[ax] += tdel[ax];
    }
    free(hist1); free(hist2); free(cur);
    return ok_cap ? emitted : -1;
}

/* ------------------------------------------------------------------------- */
/* MLP footprint model f_theta (Sec. 2.2): fully connected, SiLU between      */
/* layers, linear output.  Parameters for layer i (sizes[i] -> sizes[i+1]):   */
/* W_i [sizes[i+1]][sizes[i]] row-major, then b_i [sizes[i+1]], concatenated. */
/* act_mode 0: FP64 throughout.  act_mode 1: every weight and every hidden   */
/* activation fed to a hidden-to-hidden layer is rounded double -> float ->  */
/* bfloat16 (round to nearest even); biases, features, the first and last    */
/* layers stay at full precision: the precision contract of a BF16          */
/* tensor-core evaluation with FP32 accumulation.                            */
/* act_mode 2: as 1 but each rounded activation is carried as a pair         */
/* hi = bf16(h), lo = bf16(h - hi) (split-BF16 activations).                 */
/* ------------------------------------------------------------------------- */
static double silu(double z) { return z / (1.0 + exp(-z)); }

static double bf16_round(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f; /* inf / nan */
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

double orc_bf16_round(double x) { return bf16_round(x); }

static double act_round(double h, int mode)
{
    if (mode == 1) return bf16_round(h);
    if (mode == 2) { double hi = bf16_round(h); return hi + bf16_round((double)(float)(h - hi)); }
    return h;
}

long long orc_mlp_param_count(int nl, const int *sizes)
{
    long long t = 0;
    for (int i = 0; i < nl; ++i) t += (long long)sizes[i + 1] * sizes[i] + sizes[i + 1];
    return t;
}

/* Layers whose input and output are both hidden (0 < i < nl - 1) run on the
 * tensor cores in BF16; the first (features -> hidden) and last
 * (hidden -> scalar) layers are FP32 CUDA-core work in the kernel.  The
 * emulation rounds exactly the operands of the hidden-to-hidden layers. */
/* ov_layer >= 0: in layer ov_layer (a hidden-to-hidden layer) the input
 * activation ov_unit takes the value ov_value instead of its rounding. */
static void mlp_forward_ov(int nl, const int *sizes, const double *prm, const double *x, int mode, double *zs,
                           double *hs, double *out, int ov_layer, int ov_unit, double ov_value);

static void mlp_forward_one(int nl, const int *sizes, const double *prm, const double *x, int mode,
                            double *zs, double *hs, double *out)
{
    mlp_forward_ov(nl, sizes, prm, x, mode, zs, hs, out, -1, -1, 0.0);
}

static void mlp_forward_ov(int nl, const int *sizes, const double *prm, const double *x, int mode, double *zs,
                           double *hs, double *out, int ov_layer, int ov_unit, double ov_value)
{
    /* zs, hs: scratch of size sum(sizes[1..nl]) each; hs[0..] hidden outputs */
    const double *in = x;
    double inbuf[256];
    int in_n = sizes[0];
    for (int i = 0; i < in_n; ++i) inbuf[i] = in[i];
    const double *P = prm;
    int off = 0;
    for (int li = 0; li < nl; ++li) {
        int ni = sizes[li], no = sizes[li + 1];
        const double *Wl = P, *bl = P + (long long)no * ni;
        int tensor = (li > 0 && li < nl - 1);
        for (int o = 0; o < no; ++o) {
            double acc = 0.0;
            for (int i = 0; i < ni; ++i) {
                double wv = Wl[(long long)o * ni + i], hv = inbuf[i];
                if (mode != 0) {
                    wv = bf16_round(wv);
                    if (tensor) hv = (li == ov_layer && i == ov_unit) ? ov_value : act_round(hv, mode);
                }
                acc += wv * hv;
            }
            acc += bl[o];
            zs[off + o] = acc;
            hs[off + o] = (li == nl - 1) ? acc : silu(acc);
        }
        for (int o = 0; o < no; ++o) inbuf[o] = hs[off + o];
        off += no;
        P += (long long)no * ni + no;
    }
    *out = hs[off - 1];
}

/* The outputs of the BF16 contract (act_mode 1) with one hidden activation
 * rounded to its other BF16 neighbour: for every activation h entering a
 * hidden-to-hidden layer whose rounding changes when h moves by rel_eps |h|
 * (h lies that close to a BF16 rounding boundary), the network's output
 * with that single activation rounded the other way.  An evaluation whose
 * FP32 arithmetic puts such an activation on the other side of the
 * boundary returns one of these outputs.  Writes at most max_alts values
 * to alts and returns how many there are (possibly more than max_alts). */
long long orc_mlp_flip_variants(int nl, const int *sizes, const double *prm, const double *x, double rel_eps,
                                double *alts, long long max_alts)
{
    int tot = 0;
    for (int i = 1; i <= nl; ++i) tot += sizes[i];
    double *zs = (double *)malloc(sizeof(double) * tot), *hs = (double *)malloc(sizeof(double) * tot);
    double *zs2 = (double *)malloc(sizeof(double) * tot), *hs2 = (double *)malloc(sizeof(double) * tot);
    double base;
    mlp_forward_ov(nl, sizes, prm, x, 1, zs, hs, &base, -1, -1, 0.0);
    long long n = 0;
    int off = 0;
    for (int li = 0; li + 1 < nl; ++li) {
        const int no = sizes[li + 1];
        const int next_tensor = (li + 1 > 0 && li + 1 < nl - 1);
        for (int o = 0; o < no && next_tensor; ++o) {
            const double h = hs[off + o], r = bf16_round(h);
            const double cand[2] = {bf16_round(h - rel_eps * fabs(h)), bf16_round(h + rel_eps * fabs(h))};
            for (int c = 0; c < 2; ++c) {
                if (cand[c] == r || (c == 1 && cand[1] == cand[0])) continue;
                double v;
                mlp_forward_ov(nl, sizes, prm, x, 1, zs2, hs2, &v, li + 1, o, cand[c]);
                if (n < max_alts) alts[n] = v;
                n++;
            }
        }
        off += no;
    }
    free(zs); free(hs); free(zs2); free(hs2);
    return n;
}

void orc_mlp_forward(int nl, const int *sizes, const double *prm, long long B, const double *X, double *out, int mode)
{
    int tot = 0;
    for (int i = 1; i <= nl; ++i) tot += sizes[i];
#pragma omp parallel
    {
        double *zs = (double *)malloc(sizeof(double) * tot), *hs = (double *)malloc(sizeof(double) * tot);
#pragma omp for schedule(static)
        for (long long b = 0; b < B; ++b)
            mlp_forward_one(nl, sizes, prm, X + (long long)b * sizes[0], mode, zs, hs, out + b);
        free(zs); free(hs);
    }
}

/* Gradient of L = (1/B) sum_b (f(x_b) - y_b)^2 with respect to all
 * parameters (same layout as prm), backward in FP64.  mode 0: FP64 forward.
 * mode 1: the BF16-contract forward (act_mode 1); the backward then uses the
 * rounded weights and the rounded activations that entered each layer, and
 * passes gradients straight through the roundings.  Returns L. */
double orc_mlp_loss_grad_mode(int nl, const int *sizes, const double *prm, long long B, const double *X,
                              const double *Y, double *grad, int mode);

double orc_mlp_loss_grad(int nl, const int *sizes, const double *prm, long long B, const double *X,
                         const double *Y, double *grad)
{
    return orc_mlp_loss_grad_mode(nl, sizes, prm, B, X, Y, grad, 0);
}

double orc_mlp_loss_grad_mode(int nl, const int *sizes, const double *prm, long long B, const double *X,
                              const double *Y, double *grad, int mode)
{
    long long np = orc_mlp_param_count(nl, sizes);
    memset(grad, 0, sizeof(double) * np);
    int tot = 0, maxw = sizes[0];
    for (int i = 1; i <= nl; ++i) { tot += sizes[i]; if (sizes[i] > maxw) maxw = sizes[i]; }
    double *zs = (double *)malloc(sizeof(double) * tot), *hs = (double *)malloc(sizeof(double) * tot);
    double *g = (double *)malloc(sizeof(double) * maxw), *gn = (double *)malloc(sizeof(double) * maxw);
    long long *poff = (long long *)malloc(sizeof(long long) * (nl + 1));
    int *aoff = (int *)malloc(sizeof(int) * (nl + 1));
    poff[0] = 0; aoff[0] = 0;
    for (int i = 0; i < nl; ++i) {
        poff[i + 1] = poff[i] + (long long)sizes[i + 1] * sizes[i] + sizes[i + 1];
        aoff[i + 1] = aoff[i] + sizes[i + 1];
    }
    double loss = 0.0;
    for (long long b = 0; b < B; ++b) {
        const double *x = X + b * sizes[0];
        double f;
        mlp_forward_one(nl, sizes, prm, x, mode, zs, hs, &f);
        double r = f - Y[b];
        loss += r * r;
        /* dL/dz of the output layer */
        g[0] = 2.0 * r / (double)B;
        for (int li = nl - 1; li >= 0; --li) {
            int ni = sizes[li], no = sizes[li + 1];
            const double *Wl = prm + poff[li];
            double *gW = grad + poff[li], *gb = gW + (long long)no * ni;
            const double *hin = (li == 0) ? x : hs + aoff[li - 1];
            const int tensor = (li > 0 && li < nl - 1);
            for (int o = 0; o < no; ++o) {
                gb[o] += g[o];
                for (int i = 0; i < ni; ++i) {
                    const double hv = (mode != 0 && tensor) ? act_round(hin[i], mode) : hin[i];
                    gW[(long long)o * ni + i] += g[o] * hv;
                }
            }
            if (li == 0) break;
            /* back through W then through SiLU of the previous layer */
            for (int i = 0; i < ni; ++i) {
                double acc = 0.0;
                for (int o = 0; o < no; ++o) {
                    const double wv = mode != 0 ? bf16_round(Wl[(long long)o * ni + i]) : Wl[(long long)o * ni + i];
                    acc += wv * g[o];
                }
                double z = zs[aoff[li - 1] + i];
                double sg = 1.0 / (1.0 + exp(-z));
                gn[i] = acc * sg * (1.0 + z * (1.0 - sg));
            }
            for (int i = 0; i < ni; ++i) g[i] = gn[i];
        }
    }
    free(zs); free(hs); free(g); free(gn); free(poff); free(aoff);
    return loss / (double)B;
}

/* ------------------------------------------------------------------------- */
/* MLP input features.  The footprint is invariant under every signed        */
/* permutation G of the axes (phi is), so P_{Gw}(Gp) = P_w(p).  G maps w to  */
/* the chamber 0 <= w1 <= w2 <= w3 (flip negative components, then sort      */
/* ascending, stable).  Frame: u = normalize(e1 x w), v = u x w (Algorithm 2  */
/* only fixes u perpendicular to w and v = u x w).  Features:                 */
/* (w1, w2, w3, <Gp,u> sqrt(3)/W, <Gp,v> sqrt(3)/W): the sampling disc of     */
/* radius sqrt(3) W maps to radius 3.                                         */
/* ------------------------------------------------------------------------- */
void orc_features(int n, const double *w_in, const double *p_in, double *feat)
{
    const double W = 0.5 * (n + 1);
    double w[3], p[3];
    for (int d = 0; d < 3; ++d) {
        if (w_in[d] < 0.0) { w[d] = -w_in[d]; p[d] = -p_in[d]; }
        else { w[d] = w_in[d]; p[d] = p_in[d]; }
    }
    /* stable ascending sort of (w, p) by w (insertion sort) */
    for (int i = 1; i < 3; ++i) {
        double kw = w[i], kp = p[i];
        int j = i - 1;
        while (j >= 0 && w[j] > kw) { w[j + 1] = w[j]; p[j + 1] = p[j]; --j; }
        w[j + 1] = kw; p[j + 1] = kp;
    }
    /* u = (e1 x w)/|e1 x w| = (0, -w3, w2)/sqrt(w2^2 + w3^2) */
    double nr = sqrt(w[1] * w[1] + w[2] * w[2]);
    double u[3] = {0.0, -w[2] / nr, w[1] / nr};
    double v[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    double sc = sqrt(3.0) / W;
    feat[0] = w[0]; feat[1] = w[1]; feat[2] = w[2];
    feat[3] = (p[0] * u[0] + p[1] * u[1] + p[2] * u[2]) * sc;
    feat[4] = (p[0] * v[0] + p[1] * v[1] + p[2] * v[2]) * sc;
}

/* MLP-footprint forward: y_r = sum over the exact pair set of
 * c_k * f_theta(features(w_r, s_r - k))  (Algorithm 2 with f_theta, output
 * kept only on the exact support of the basis). */
typedef struct {
    int n, nl; const int *sizes; const double *prm; int mode; const double *w; const double *c;
    double sum; double *zs, *hs;
} mlpf_ctx;

static void mlpf_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    mlpf_ctx *x = (mlpf_ctx *)vctx;
    double f[5], o;
    orc_features(x->n, x->w, p, f);
    if (x->mode != 0) for (int i = 0; i < 5; ++i) f[i] = (double)(float)f[i];
    mlp_forward_one(x->nl, x->sizes, x->prm, f, x->mode, x->zs, x->hs, &o);
    x->sum += x->c[kidx] * o;
}

void orc_forward_mlp(int n, const int *dims, const double *org, const double *c, const orc_geom *g,
                     int nl, const int *sizes, const double *prm, int mode, double *y)
{
    long long nr = orc_geom_rays(g);
    int tot = 0;
    for (int i = 1; i <= nl; ++i) tot += sizes[i];
#pragma omp parallel
    {
        double *zs = (double *)malloc(sizeof(double) * tot), *hs = (double *)malloc(sizeof(double) * tot);
#pragma omp for schedule(dynamic, 4)
        for (long long r = 0; r < nr; ++r) {
            double s[3], w[3];
            orc_geom_ray(g, r, s, w);
            mlpf_ctx x = {n, nl, sizes, prm, mode, w, c, 0.0, zs, hs};
            for_each_pair(n, dims, org, s, w, mlpf_visit, &x);
            y[r] = x.sum;
        }
        free(zs); free(hs);
    }
}

/* ------------------------------------------------------------------------- */
/* Footprint tables (the splat form: an approximation of Eq. 4's            */
/* contribution).  For a parallel view the direction w is fixed, so the      */
/* footprint is one 2-D function on H_w.  With the orthonormal frame         */
/* e1 = (u - (u.w) w) / |u - (u.w) w| (u = det_u of the view), e2 = w x e1,  */
/* it is tabulated exactly at the nodes (i - M) h e1 + (j - M) h e2,         */
/* i, j = 0..2M, M = ceil(sqrt(3) W / h) + 1 (the disc of radius sqrt(3) W   */
/* that holds the cube's shadow, one node of margin), and the footprint of   */
/* a pair is the bilinear interpolation of the table at the pair's offset,   */
/* zero outside the table.  The pairs are the exact ones (for_each_pair).    */
/* ------------------------------------------------------------------------- */
int orc_table_radius(int n, double h) { return (int)ceil(sqrt(3.0) * 0.5 * (n + 1) / h) + 1; }

void orc_table_frame(const double *dir, const double *du, double *w, double *e1, double *e2)
{
    double nw = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    for (int d = 0; d < 3; ++d) w[d] = dir[d] / nw;
    double uw = du[0] * w[0] + du[1] * w[1] + du[2] * w[2];
    double e[3], ne = 0.0;
    for (int d = 0; d < 3; ++d) { e[d] = du[d] - uw * w[d]; ne += e[d] * e[d]; }
    ne = sqrt(ne);
    for (int d = 0; d < 3; ++d) e1[d] = e[d] / ne;
    e2[0] = w[1] * e1[2] - w[2] * e1[1];
    e2[1] = w[2] * e1[0] - w[0] * e1[2];
    e2[2] = w[0] * e1[1] - w[1] * e1[0];
}

double orc_table_footprint(int n, const double *w, const double *e1, const double *e2, double h, const double *p)
{
    const int M = orc_table_radius(n, h);
    const double a = (p[0] * e1[0] + p[1] * e1[1] + p[2] * e1[2]) / h + M;
    const double b = (p[0] * e2[0] + p[1] * e2[1] + p[2] * e2[2]) / h + M;
    const double ia = floor(a), ib = floor(b);
    if (ia < 0.0 || ib < 0.0 || ia + 1.0 > 2.0 * M || ib + 1.0 > 2.0 * M) return 0.0;
    const double ta = a - ia, tb = b - ib;
    double v[2][2];
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj) {
            double q[3];
            for (int d = 0; d < 3; ++d) q[d] = (ia + di - M) * h * e1[d] + (ib + dj - M) * h * e2[d];
            v[di][dj] = orc_footprint(n, w, q);
        }
    return (1.0 - ta) * (1.0 - tb) * v[0][0] + ta * (1.0 - tb) * v[1][0] + (1.0 - ta) * tb * v[0][1] +
           ta * tb * v[1][1];
}

typedef struct { int n; const double *w, *e1, *e2; double h; const double *c; double yr; double *cout; double sum; } tab_ctx;

static void tabf_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    tab_ctx *x = (tab_ctx *)vctx;
    x->sum += x->c[kidx] * orc_table_footprint(x->n, x->w, x->e1, x->e2, x->h, p);
}

static void taba_visit(void *vctx, long long kidx, const int *k, const double *p)
{
    (void)k;
    tab_ctx *x = (tab_ctx *)vctx;
    x->cout[kidx] += x->yr * orc_table_footprint(x->n, x->w, x->e1, x->e2, x->h, p);
}

/* the view of ray r of a parallel geometry and its table frame */
static void table_ray(const orc_geom *g, long long r, double *s, double *w, double *e1, double *e2)
{
    double ww[3];
    orc_geom_ray(g, r, s, ww);
    const int v = (int)(r / ((long long)g->nu * g->nv));
    orc_table_frame(g->dir_or_src + 3 * v, g->det_u + 3 * v, w, e1, e2);
}

/* y = A_T c over the exact pair set (parallel geometries only) */
void orc_forward_table(int n, const int *dims, const double *org, const double *c, const orc_geom *g, double h,
                       double *y)
{
    long long nr = orc_geom_rays(g);
#pragma omp parallel for schedule(dynamic, 4)
    for (long long r = 0; r < nr; ++r) {
        double s[3], w[3], e1[3], e2[3];
        table_ray(g, r, s, w, e1, e2);
        tab_ctx x = {n, w, e1, e2, h, c, 0.0, NULL, 0.0};
        for_each_pair(n, dims, org, s, w, tabf_visit, &x);
        y[r] = x.sum;
    }
}

/* c = A_T^T y (transpose of the same matrix), overwrites c; serial scatter */
void orc_adjoint_table(int n, const int *dims, const double *org, const double *y, const orc_geom *g, double h,
                       double *c)
{
    long long nk = (long long)dims[0] * dims[1] * dims[2], nr = orc_geom_rays(g);
    memset(c, 0, sizeof(double) * nk);
    for (long long r = 0; r < nr; ++r) {
        if (y[r] == 0.0) continue;
        double s[3], w[3], e1[3], e2[3];
        table_ray(g, r, s, w, e1, e2);
        tab_ctx x = {n, w, e1, e2, h, NULL, y[r], c, 0.0};
        for_each_pair(n, dims, org, s, w, taba_visit, &x);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
