// geometry.cu -- geometry objects (Eq. 1 lines on the device), error
// reporting and the Gauss-Legendre rule of libspl.so.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "spl_host.h"

namespace spl {

static thread_local char g_last_error[512] = "";

spl_status fail(spl_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_last_error[0] = '\0'; }

spl_status cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SPL_OK;
    return fail(SPL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- per-device state
namespace {
constexpr int kMaxDev = 64;
std::mutex g_dev_mutex;
int g_sm_count[kMaxDev];             // 0: not queried yet
struct AttrDone {
    const void *func;
    int device;
};
AttrDone g_attr_done[256];
int g_attr_n = 0;
}  // namespace

int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (g_sm_count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 1;
        }
        g_sm_count[dev] = n;
    }
    return g_sm_count[dev];
}

spl_status smem_attr_once(const void *func, int bytes, const char *what)
{
    int dev = 0;
    spl_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != SPL_OK) return s;
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    for (int i = 0; i < g_attr_n; ++i)
        if (g_attr_done[i].func == func && g_attr_done[i].device == dev) return SPL_OK;
    s = cuda_check(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), what);
    if (s != SPL_OK) return s;
    if (g_attr_n < (int)(sizeof(g_attr_done) / sizeof(g_attr_done[0]))) g_attr_done[g_attr_n++] = {func, dev};
    return SPL_OK;
}

// ---------------------------------------------------------------- quadrature
// Roots of the Legendre polynomial P_m by Newton's method from Tricomi's
// asymptotic initial guess, in long double; weights 2/((1-x^2) P_m'(x)^2).
static void legendre_rule(int m, double *x, double *w)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < m; ++i) {
        const long double th = pi * (4.0L * (i + 1) - 1.0L) / (4.0L * m + 2.0L);
        long double z = (1.0L - (m - 1.0L) / (8.0L * m * m * m)) * cosl(th);
        long double dp = 1.0L;
        for (int it = 0; it < 64; ++it) {
            long double pk = z, pkm1 = 1.0L;  // P_1, P_0
            for (int k = 1; k < m; ++k) {
                const long double pk1 = ((2.0L * k + 1.0L) * z * pk - k * pkm1) / (k + 1.0L);
                pkm1 = pk;
                pk = pk1;
            }
            if (m == 1) { pk = z; pkm1 = 1.0L; }
            dp = m * (pkm1 - z * pk) / (1.0L - z * z);
            const long double step = pk / dp;
            z -= step;
            if (fabsl(step) < 1e-19L) break;
        }
        x[i] = (double)z;
        w[i] = (double)(2.0L / ((1.0L - z * z) * dp * dp));
    }
}

static QuadRule g_rules[4];
static int g_iter_cap = kIterCap;
static std::once_flag g_rules_once;

static void init_rules()
{
    for (int n = 0; n < 4; ++n) {
        const int m = (3 * n + 2) / 2 > 0 ? (3 * n + 2) / 2 : 1;
        double x[kMaxNodes], w[kMaxNodes];
        legendre_rule(m, x, w);
        for (int q = 0; q < kMaxNodes; ++q) {
            g_rules[n].x[q] = q < m ? (float)x[q] : 0.0f;
            g_rules[n].w[q] = q < m ? (float)w[q] : 0.0f;
        }
        // n+1 nodes: exact for the degree-2n products of flat rays
        legendre_rule(n + 1, x, w);
        for (int q = 0; q < kMaxNodes; ++q) {
            g_rules[n].x1[q] = q <= n ? (float)x[q] : 0.0f;
            g_rules[n].w1[q] = q <= n ? (float)w[q] : 0.0f;
        }
    }
}

QuadRule quad_rule(int degree)
{
    std::call_once(g_rules_once, init_rules);
    QuadRule q = g_rules[degree];
    q.cap = g_iter_cap;
    return q;
}

int set_iter_cap(int cap)
{
    const int old = g_iter_cap;
    g_iter_cap = (cap < 1 || cap > kIterCap) ? kIterCap : cap;
    return old;
}

int quad_nodes(int degree) { return (3 * degree + 2) / 2 > 0 ? (3 * degree + 2) / 2 : 1; }

spl_status check_basis(const spl_basis_desc *b)
{
    if (!b) return fail(SPL_ERR_ARG, "basis descriptor is NULL");
    if (b->degree < 0 || b->degree > 3) return fail(SPL_ERR_ARG, "degree %d not in 0..3", b->degree);
    if (b->mode != SPL_FP_QUAD && b->mode != SPL_FP_MLP && b->mode != SPL_FP_DIRECT && b->mode != SPL_FP_TABLE)
        return fail(SPL_ERR_ARG, "unknown footprint mode %d", b->mode);
    if (b->mode == SPL_FP_MLP && !b->mlp) return fail(SPL_ERR_ARG, "SPL_FP_MLP needs an MLP");
    if (b->separable != SPL_SEP_AUTO && b->separable != SPL_SEP_OFF)
        return fail(SPL_ERR_ARG, "unknown separable mode %d", b->separable);
    return SPL_OK;
}

}  // namespace spl

using namespace spl;

static bool finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Slice-separable view (see spl_prepare in spl.h): the direction's zero
// component is the b axis of its direction set-up, det_u has no b
// component and det_v only a b component.  Key of a group: b, and the b
// index coordinate of detector row v, z0 + v dz.
struct SepKey {
    int b;
    double z0, dz;
};

static bool sep_of(const ViewPose &P, const double *origin, int nv, SepKey &k)
{
    const int b = P.dir.ax[2];
    if (P.dir.r[1] != 0.0 || P.du[b] != 0.0 || P.dv[b] == 0.0) return false;
    for (int e = 0; e < 3; ++e)
        if (e != b && P.dv[e] != 0.0) return false;
    k.b = b;
    k.dz = P.dv[b];
    k.z0 = P.dc[b] - origin[b] - 0.5 * (nv - 1) * P.dv[b];
    return true;
}

static bool sep_key_of(const ViewPose &P, const double *origin, int nv, const SepKey &key)
{
    SepKey k;
    return sep_of(P, origin, nv, k) && k.b == key.b && k.z0 == key.z0 && k.dz == key.dz;
}

// the largest group among the first few distinct keys; returns its size
static int separable_group(const ViewPose *views, int n_views, const double *origin, int nv, SepKey &best)
{
    constexpr int kKeys = 8;
    SepKey keys[kKeys];
    int cnt[kKeys] = {0}, nk = 0;
    for (int v = 0; v < n_views; ++v) {
        SepKey k;
        if (!sep_of(views[v], origin, nv, k)) continue;
        int i = 0;
        while (i < nk && !(keys[i].b == k.b && keys[i].z0 == k.z0 && keys[i].dz == k.dz)) ++i;
        if (i == nk) {
            if (nk == kKeys) continue;
            keys[nk++] = k;
        }
        ++cnt[i];
    }
    int bi = -1;
    for (int i = 0; i < nk; ++i)
        if (bi < 0 || cnt[i] > cnt[bi]) bi = i;
    if (bi < 0) return 0;
    best = keys[bi];
    return cnt[bi];
}

extern "C" spl_status spl_make_geometry(const spl_geometry_desc *desc, spl_geometry **out)
{
    clear_error();
    if (!out) return fail(SPL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(SPL_ERR_ARG, "desc is NULL");
    const spl_geometry_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > 2048 || d.ny > 2048 || d.nz > 2048)
        return fail(SPL_ERR_UNSUPPORTED, "grid %d x %d x %d outside 1..2048 per axis", d.nx, d.ny, d.nz);
    if ((long long)d.nx * d.ny * d.nz >= (1LL << 31)) return fail(SPL_ERR_UNSUPPORTED, "grid has 2^31 or more coefficients");
    if (!finite3(d.origin)) return fail(SPL_ERR_NONFINITE, "origin is not finite");

    spl_geometry *g = (spl_geometry *)calloc(1, sizeof(spl_geometry));
    if (!g) return fail(SPL_ERR_OOM, "host allocation failed");
    g->desc = d;
    g->desc.ray_omega = g->desc.ray_s = nullptr;
    g->desc.view_src = g->desc.det_center = g->desc.det_u = g->desc.det_v = nullptr;
    DevGeom &dg = g->dev;
    dg.kind = d.kind;
    dg.n[0] = d.nx;
    dg.n[1] = d.ny;
    dg.n[2] = d.nz;
    for (int e = 0; e < 3; ++e) dg.org[e] = d.origin[e];
    size_t payload = 0;
    double *ray_host = nullptr;
    int *view_order = nullptr;
    size_t order_off = 0;

    if (d.kind == SPL_RAYS) {
        if (d.n_rays < 0 || (d.n_rays > 0 && (!d.ray_omega || !d.ray_s))) {
            free(g);
            return fail(SPL_ERR_ARG, "rays: bad count or NULL arrays");
        }
        dg.n_rays = d.n_rays;
        payload = (size_t)d.n_rays * 6 * sizeof(double);
        ray_host = (double *)malloc(payload > 0 ? payload : 1);
        if (!ray_host) { free(g); return fail(SPL_ERR_OOM, "host allocation failed"); }
        for (long long r = 0; r < d.n_rays; ++r) {
            const double *w = d.ray_omega + 3 * r, *s = d.ray_s + 3 * r;
            if (!finite3(w) || !finite3(s)) { free(ray_host); free(g); return fail(SPL_ERR_NONFINITE, "ray %lld is not finite", r); }
            const double nrm = sqrt(dot3(w, w));
            if (!(nrm > 0.0) || !isfinite(nrm)) { free(ray_host); free(g); return fail(SPL_ERR_NONFINITE, "ray %lld has a zero direction", r); }
            for (int e = 0; e < 3; ++e) {
                ray_host[3 * r + e] = w[e] / nrm;                 // directions first
                ray_host[3 * d.n_rays + 3 * r + e] = s[e];        // then points
            }
        }
    } else if (d.kind == SPL_PARALLEL || d.kind == SPL_CONE) {
        if (d.n_views < 0 || d.n_views > 65535 || d.nu < 1 || d.nv < 1 || d.nu > 65535 || d.nv > 65535 ||
            (d.n_views > 0 && (!d.view_src || !d.det_center || !d.det_u || !d.det_v))) {
            free(g);
            return fail(SPL_ERR_ARG, "views: bad counts (views <= 65535, pixels >= 1) or NULL arrays");
        }
        dg.n_views = d.n_views;
        dg.nu = d.nu;
        dg.nv = d.nv;
        dg.n_rays = (long long)d.n_views * d.nu * d.nv;
        g->views_host = (ViewPose *)calloc(d.n_views > 0 ? d.n_views : 1, sizeof(ViewPose));
        if (!g->views_host) { free(g); return fail(SPL_ERR_OOM, "host allocation failed"); }
        for (int k = 0; k < d.n_views; ++k) {
            ViewPose &P = g->views_host[k];
            const double *src = d.view_src + 3 * k;
            for (int e = 0; e < 3; ++e) {
                P.src[e] = src[e];
                P.dc[e] = d.det_center[3 * k + e];
                P.du[e] = d.det_u[3 * k + e];
                P.dv[e] = d.det_v[3 * k + e];
            }
            if (!finite3(P.src) || !finite3(P.dc) || !finite3(P.du) || !finite3(P.dv)) {
                free(g->views_host); free(g);
                return fail(SPL_ERR_NONFINITE, "view %d is not finite", k);
            }
            double n[3];
            cross3(P.du, P.dv, n);
            const double nn = sqrt(dot3(n, n));
            if (!(nn > 0.0)) { free(g->views_host); free(g); return fail(SPL_ERR_NONFINITE, "view %d: detector axes are parallel", k); }
            for (int e = 0; e < 3; ++e) P.nrm[e] = n[e] / nn;
            // dual axes of (du, dv) in the detector plane: ud = (dv x n)/det, vd = (n x du)/det
            double t1[3], t2[3];
            cross3(P.dv, P.nrm, t1);
            cross3(P.nrm, P.du, t2);
            const double det = dot3(P.du, t1);
            for (int e = 0; e < 3; ++e) {
                P.ud[e] = t1[e] / det;
                P.vd[e] = t2[e] / det;
            }
            if (d.kind == SPL_PARALLEL) {
                const double l = sqrt(dot3(P.src, P.src));
                if (!(l > 0.0)) { free(g->views_host); free(g); return fail(SPL_ERR_NONFINITE, "view %d: zero direction", k); }
                for (int e = 0; e < 3; ++e) P.src[e] /= l;
                dir_setup(P.src, P.dir);
                // footprint-table frame: det_u without its w component, and w x e1
                double e[3];
                const double uw = dot3(P.du, P.src);
                for (int q = 0; q < 3; ++q) e[q] = P.du[q] - uw * P.src[q];
                const double ne = sqrt(dot3(e, e));
                if (!(ne > 0.0)) {
                    free(g->views_host); free(g);
                    return fail(SPL_ERR_ARG, "view %d: det_u is parallel to the ray direction", k);
                }
                for (int q = 0; q < 3; ++q) P.e1[q] = e[q] / ne;
                cross3(P.src, P.e1, P.e2);
                if (fabs(dot3(P.src, P.nrm)) < 1e-12) {
                    free(g->views_host); free(g);
                    return fail(SPL_ERR_ARG, "view %d: ray direction lies in the detector plane", k);
                }
            } else {
                // every pixel must be at a positive distance from the source
                double rel[3];
                for (int e = 0; e < 3; ++e) rel[e] = P.dc[e] - P.src[e];
                if (!(fabs(dot3(rel, P.nrm)) > 0.0)) {
                    free(g->views_host); free(g);
                    return fail(SPL_ERR_ARG, "view %d: source lies in the detector plane", k);
                }
            }
        }
        payload = (size_t)d.n_views * sizeof(ViewPose);
        if (d.kind == SPL_PARALLEL) {
            // view order: the slice-separable group, the other views whose
            // rays have a zero transverse component (flat march), the rest;
            // each class gets its own launch
            view_order = (int *)malloc((d.n_views > 0 ? d.n_views : 1) * sizeof(int));
            if (!view_order) { free(g->views_host); free(g); return fail(SPL_ERR_OOM, "host allocation failed"); }
            SepKey key;
            const int n_sep = separable_group(g->views_host, d.n_views, d.origin, d.nv, key);
            int n = 0;
            for (int k = 0; k < d.n_views; ++k)
                if (n_sep > 0 && sep_key_of(g->views_host[k], d.origin, d.nv, key)) view_order[n++] = k;
            for (int k = 0; k < d.n_views; ++k)
                if (g->views_host[k].dir.rb == 0.0f && !(n_sep > 0 && sep_key_of(g->views_host[k], d.origin, d.nv, key)))
                    view_order[n++] = k;
            dg.n_flat = n;
            for (int k = 0; k < d.n_views; ++k)
                if (g->views_host[k].dir.rb != 0.0f) view_order[n++] = k;
            dg.n_sep = n_sep;
            if (n_sep > 0) {
                PlaneGroup *pg = new PlaneGroup();
                pg->b = key.b;
                pg->p = key.b == 0 ? 1 : 0;
                pg->q = key.b == 2 ? 1 : 2;
                pg->n_views = n_sep;
                pg->rows = (long long)n_sep * d.nu;
                pg->ncol = (long long)dg.n[pg->p] * dg.n[pg->q];
                pg->z0 = key.z0;
                pg->dz = key.dz;
                pg->side = nullptr;
                pg->fork = pg->join = nullptr;
                if (cudaStreamCreateWithFlags(&pg->side, cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&pg->fork, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&pg->join, cudaEventDisableTiming) != cudaSuccess) {
                    cudaGetLastError();
                    if (pg->fork) cudaEventDestroy(pg->fork);
                    if (pg->side) cudaStreamDestroy(pg->side);
                    pg->side = nullptr;
                    pg->fork = pg->join = nullptr;
                }
                g->plane = pg;
            }
            g->vconst = (ViewConst *)malloc((d.n_views > 0 ? d.n_views : 1) * sizeof(ViewConst));
            if (!g->vconst) {
                free(view_order);
                plane_free(g->plane);
                free(g->views_host);
                free(g);
                return fail(SPL_ERR_OOM, "host allocation failed");
            }
            for (int i = 0; i < d.n_views; ++i) {
                const ViewPose &P = g->views_host[view_order[i]];
                view_const(P.dir, view_order[i], dg.n, g->vconst[i]);
                view_const_frame(P.dir, P.e1, P.e2, g->vconst[i]);
            }
            order_off = (payload + 255) & ~(size_t)255;
            payload = order_off + (size_t)d.n_views * sizeof(int);
        }
    } else {
        free(g);
        return fail(SPL_ERR_ARG, "unknown geometry kind %d", d.kind);
    }

    cudaGetDevice(&g->device);
    // the caller's arrays as given (the exact pair count rebuilds rays from them)
    const size_t raw_off = (payload + 255) & ~(size_t)255;
    const size_t raw_bytes = d.kind == SPL_RAYS ? (size_t)d.n_rays * 6 * sizeof(double)
                                                : (size_t)d.n_views * 12 * sizeof(double);
    double *raw_host = (double *)malloc(raw_bytes > 0 ? raw_bytes : 1);
    if (!raw_host) {
        free(ray_host);
        free(view_order);
        plane_free(g->plane);
        free(g->vconst);
        free(g->views_host);
        free(g);
        return fail(SPL_ERR_OOM, "host allocation failed");
    }
    if (d.kind == SPL_RAYS) {
        for (long long r = 0; r < d.n_rays; ++r)
            for (int e = 0; e < 3; ++e) {
                raw_host[6 * r + e] = d.ray_omega[3 * r + e];
                raw_host[6 * r + 3 + e] = d.ray_s[3 * r + e];
            }
    } else {
        for (int k = 0; k < d.n_views; ++k)
            for (int e = 0; e < 3; ++e) {
                raw_host[12 * k + e] = d.view_src[3 * k + e];
                raw_host[12 * k + 3 + e] = d.det_center[3 * k + e];
                raw_host[12 * k + 6 + e] = d.det_u[3 * k + e];
                raw_host[12 * k + 9 + e] = d.det_v[3 * k + e];
            }
    }
    const size_t flag_off = (raw_off + raw_bytes + 255) & ~(size_t)255;
    void *blk = nullptr;
    cudaError_t ce = cudaMalloc(&blk, flag_off + 256);
    if (ce != cudaSuccess) {
        free(raw_host);
        free(ray_host);
        free(view_order);
        plane_free(g->plane);
        free(g->vconst);
        free(g->views_host);
        free(g);
        cudaGetLastError();
        return fail(SPL_ERR_OOM, "cudaMalloc(%zu) failed: %s", flag_off + 256, cudaGetErrorString(ce));
    }
    g->dev_block = blk;
    const void *src = d.kind == SPL_RAYS ? (const void *)ray_host : (const void *)g->views_host;
    const size_t src_bytes = view_order ? (size_t)d.n_views * sizeof(ViewPose) : payload;
    if (src_bytes > 0) ce = cudaMemcpy(blk, src, src_bytes, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && view_order && d.n_views > 0)
        ce = cudaMemcpy((char *)blk + order_off, view_order, (size_t)d.n_views * sizeof(int), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && raw_bytes > 0) ce = cudaMemcpy((char *)blk + raw_off, raw_host, raw_bytes, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset((char *)blk + flag_off, 0, 256);
    free(raw_host);
    free(ray_host);
    free(view_order);
    if (ce != cudaSuccess) {
        cudaFree(blk);
        plane_free(g->plane);
        free(g->vconst);
        free(g->views_host);
        free(g);
        return cuda_check(ce, "geometry upload");
    }
    if (d.kind == SPL_RAYS) {
        dg.ray_w = (const double *)blk;
        dg.ray_s = (const double *)blk + 3 * d.n_rays;
    } else {
        dg.views = (const ViewPose *)blk;
        if (d.kind == SPL_PARALLEL) dg.view_order = (const int *)((const char *)blk + order_off);
    }
    dg.raw = (const double *)((const char *)blk + raw_off);
    dg.err = (int *)((char *)blk + flag_off);
    // The scatter adjoint of a geometry with more than one batch of views
    // (rays) adds the batches in an FP64 accumulator of the grid's size
    // (scratch sized here, so the adjoint itself allocates nothing).
    const long long nk = (long long)dg.n[0] * dg.n[1] * dg.n[2];
    const bool batched = d.kind == SPL_RAYS ? dg.n_rays > kAdjBatchRays : d.n_views > kAdjBatchViews;
    g->acc64 = nullptr;
    if (batched && dg.n_rays > 0) {
        ce = cudaMalloc((void **)&g->acc64, (size_t)nk * sizeof(double));
        if (ce != cudaSuccess) {
            cudaGetLastError();
            g->acc64 = nullptr;
            cudaFree(blk);
            plane_free(g->plane);
            free(g->vconst);
            free(g->views_host);
            free(g);
            return fail(SPL_ERR_OOM, "cudaMalloc of the adjoint accumulator (%lld doubles) failed", nk);
        }
    }
    // the scatter adjoint reduces each piece-marched ray into the layout of
    // c whose contiguous axis is the ray's b axis, kept as four copies
    // shifted by 0..3 floats (copy stride lay_cs, a multiple of 4 that
    // holds nk + 3 floats): scratch of the geometry, folded into c after
    // each batch; parallel geometries need it only for views outside the
    // flat class
    g->lay[0] = g->lay[1] = g->lay[2] = nullptr;
    g->dev.lay_cs = ((size_t)nk + 6) & ~(size_t)3;
    if (dg.n_rays > 0 && (d.kind != SPL_PARALLEL || dg.n_flat < dg.n_views)) {
        for (int L = 0; L < 3; ++L) {
            ce = cudaMalloc((void **)&g->lay[L], 4 * g->dev.lay_cs * sizeof(float));
            if (ce == cudaSuccess) ce = cudaMemset(g->lay[L], 0, 4 * g->dev.lay_cs * sizeof(float));
            if (ce != cudaSuccess) {
                cudaGetLastError();
                for (int M = 0; M <= L; ++M)
                    if (g->lay[M]) cudaFree(g->lay[M]);
                if (g->acc64) cudaFree(g->acc64);
                cudaFree(blk);
                plane_free(g->plane);
                free(g->vconst);
                free(g->views_host);
                free(g);
                return fail(SPL_ERR_OOM, "cudaMalloc of the adjoint's layout copies (4 x %lld floats) failed", nk);
            }
        }
    }
    *out = g;
    return SPL_OK;
}

extern "C" void spl_destroy_geometry(spl_geometry *g)
{
    if (!g) return;
    plane_free(g->plane);
    table_free(g->table);
    free(g->vconst);
    if (g->acc64) cudaFree(g->acc64);
    for (int L = 0; L < 3; ++L)
        if (g->lay[L]) cudaFree(g->lay[L]);
    if (g->dev_block) cudaFree(g->dev_block);
    free(g->views_host);
    free(g);
}

extern "C" long long spl_geometry_rays(const spl_geometry *g) { return g ? g->dev.n_rays : -1; }

extern "C" long long spl_geometry_coeffs(const spl_geometry *g)
{
    return g ? (long long)g->dev.n[0] * g->dev.n[1] * g->dev.n[2] : -1;
}

extern "C" spl_status spl_geometry_status(const spl_geometry *g, void *stream)
{
    clear_error();
    if (!g) return fail(SPL_ERR_ARG, "geometry is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    spl_status s = cuda_check(cudaMemcpyAsync(&flag, g->dev.err, sizeof(int), cudaMemcpyDeviceToHost, st), "status read");
    if (s != SPL_OK) return s;
    s = cuda_check(cudaStreamSynchronize(st), "status sync");
    if (s != SPL_OK) return s;
    if (flag) {
        s = cuda_check(cudaMemsetAsync(g->dev.err, 0, sizeof(int), st), "status clear");
        if (s != SPL_OK) return s;
        cudaStreamSynchronize(st);
        if (flag & 2) return fail(SPL_ERR_TIMEOUT, "a bounded tensor-core wait gave up (flag 0x%x)", flag);
        return fail(SPL_ERR_STEPCAP, "a kernel reached a loop bound (flag 0x%x)", flag);
    }
    return SPL_OK;
}

extern "C" const char *spl_last_error(void) { return spl::g_last_error; }

extern "C" int spl_debug_set_iter_cap(int cap) { return spl::set_iter_cap(cap); }

extern "C" const char *spl_version(void) { return "libspl 0.1 (sm_103a)"; }
