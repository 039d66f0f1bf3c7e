// table.cu -- footprint tables: the splat form of the footprint (SPL_FP_TABLE).
//
// For a parallel view the direction w is fixed, so the footprint of Eq. 4 is
// one 2-D function on H_w.  It is tabulated once per view and degree at the
// nodes (i - M) h e1 + (j - M) h e2 (i, j = 0..2M, h = 1/32, M =
// ceil(sqrt(3) W / h) + 1: the disc of radius sqrt(3) W that holds the cube's
// shadow, one node of margin), with (e1, e2) an orthonormal frame of H_w
// (e1 = det_u without its w component, e2 = w x e1), by the exact footprint
// evaluator.  A pair's footprint is then the bilinear interpolation of the
// table at the pair's offset: an approximation (second order in h) that
// needs no quadrature at all.
//
// The rays are walked with the same cells and knot crossings as the exact
// march, but nothing is integrated: the bases whose support the ray crosses
// are exactly those that enter the (n+1)^3 window (at the start of the ray
// or at an event), so each is looked up once, when it enters.  The offset of
// the window's base basis in (e1, e2) is carried as a double-float pair and
// stepped with the window, so a lookup position is exact to ~1e-7.
// Forward: y_r = sum c_l P_table; adjoint: c_l += y_r P_table (float atomics).
#include <math.h>
#include <string.h>

#include <mutex>

#include "spl_footprint.cuh"
#include "spl_host.h"

namespace spl {

constexpr double kTableStep = 1.0 / 32.0;

static int table_radius(int n) { return (int)ceil(sqrt(3.0) * 0.5 * (n + 1) / kTableStep) + 1; }

struct TablePack {
    int state;  // 0 not built, 1 built, -1 unavailable
    float *T;   // [n_views][2M+1][2M+1], view in the geometry's order
    int M;
};

struct TableSet {
    TablePack pack[4];
};

// one thread per table node of one view
template <int N>
__global__ void __launch_bounds__(128) k_table_build(DevGeom g, int M, double h, float *T, QuadRule qr)
{
    const long long side = 2LL * M + 1, per = side * side;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= per * g.n_views) return;
    const int k = (int)(idx / per);
    const long long r = idx - (long long)k * per;
    const int i = (int)(r / side), j = (int)(r - (long long)i * side);
    const ViewPose &P = g.views[k];
    double w[3], q[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        w[e] = P.src[e];
        q[e] = (i - M) * h * P.e1[e] + (j - M) * h * P.e2[e];
    }
    T[idx] = footprint_exact<N>(w, q, qr);
}

// (h, l) -= (dh, dl) as double-float pairs (TwoSum, renormalised)
__device__ __forceinline__ void df_sub(float &h, float &l, float dh, float dl)
{
    const float s = __fsub_rn(h, dh);
    const float bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(-dh, bb));
    const float lo = __fadd_rn(__fsub_rn(l, dl), err);
    h = __fadd_rn(s, lo);
    l = __fsub_rn(lo, __fsub_rn(h, s));
}

// Walk one ray and look every entering basis up in the view's table Tv.
// (ah, al), (bh, bl): offset of the window's base basis (c - N, QA - N,
// QB - N) in (e1, e2).  Returns false if a bound was reached.
template <int N, bool ADJ>
__device__ __forceinline__ bool table_march(const RaySetup &rs, const ViewConst &V, double al0, double be0,
                                            const float *__restrict__ Tv, int M, float inv_h,
                                            const float *__restrict__ cin,
                                            float *__restrict__ cout, float yr, const QuadRule &qr, bool kahan,
                                            float &out)
{
    out = 0.0f;
    int c = rs.c0;
    const int cl = rs.c1;
    if (c > cl) return true;
    const int side = 2 * M + 1;
    const float fM = (float)M;
    const SinkBox bx = make_box(rs.lo, rs.hi);
    int IA, IB, IAn, IBn;
    float fa, fb, fan, fbn;
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c - rs.c0, IA, fa);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c - rs.c0, IB, fb);
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
    int QA = IA, QB = IB;
    float ah, al, bh, bl;
    {
        double e1[3], e2[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            e1[q] = (double)V.E1h[q] + (double)V.E1l[q];
            e2[q] = (double)V.E2h[q] + (double)V.E2l[q];
        }
        const double a = al0 - ((c - N) * e1[0] + (QA - N) * e1[1] + (QB - N) * e1[2]);
        const double b = be0 - ((c - N) * e2[0] + (QA - N) * e2[1] + (QB - N) * e2[2]);
        ah = (float)a;
        al = (float)(a - (double)ah);
        bh = (float)b;
        bl = (float)(b - (double)bh);
    }
    float acc = 0.0f, sum = 0.0f, comp = 0.0f;
    // basis (c - N + d, QA - N + i, QB - N + k): table footprint, then its
    // contribution
    auto visit = [&](int d, int i, int k) {
        const int ld = c - N + d, la = QA - N + i, lb = QB - N + k;
        const float a = ah + (al - (d * V.E1h[0] + i * V.E1h[1] + k * V.E1h[2]));
        const float b = bh + (bl - (d * V.E2h[0] + i * V.E2h[1] + k * V.E2h[2]));
        const float pa = fmaf(a, inv_h, fM), pb = fmaf(b, inv_h, fM);
        const float ia = floorf(pa), ib = floorf(pb);
        float P = 0.0f;
        if (ia >= 0.0f && ib >= 0.0f && ia < 2.0f * fM && ib < 2.0f * fM) {
            const float ta = pa - ia, tb = pb - ib;
            const float *t = Tv + ((int)ia * side + (int)ib);
            const float lo = fmaf(tb, __ldg(t + 1) - __ldg(t), __ldg(t));
            const float hi = fmaf(tb, __ldg(t + side + 1) - __ldg(t + side), __ldg(t + side));
            P = fmaf(ta, hi - lo, lo);
        }
        if (bx.in0(ld) && bx.in1(la) && bx.in2(lb)) {
            const unsigned o = (unsigned)ld * (unsigned)rs.S[0] + (unsigned)la * (unsigned)rs.S[1] +
                               (unsigned)lb * (unsigned)rs.S[2];
            if (ADJ) {
                if (P != 0.0f) atomicAdd(cout + o, yr * P);
            } else {
                acc = fmaf(__ldg(cin + o), P, acc);
            }
        }
    };
    // the bases live at the start of the ray
#pragma unroll
    for (int d = 0; d <= N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k <= N; ++k) visit(d, i, k);
    int na = IAn - QA, nb = IBn - QB;
    if (na > 2 || nb > 2) return false;
    float ga = fa, gb = fb;
    float ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
    float tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
    int ev_in_cell = 0;
#pragma unroll 1
    while (true) {
        const bool evA = ta <= tb && ta <= 1.0f;
        const bool evB = !evA && tb <= 1.0f;
        const bool evD = !evA && !evB;
        if (evA) {
            ++QA;
            ga -= 1.0f;
            ta = --na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
        } else if (evB) {
            ++QB;
            gb -= 1.0f;
            tb = --nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
        } else {
            if (++c > cl) break;
            IA = IAn;
            fa = fan;
            IB = IBn;
            fb = fbn;
            df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
            df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
            na = IAn - QA;
            nb = IBn - QB;
            if (na > 2 || nb > 2) return false;
            ga = (float)(IA - QA) + fa;
            gb = (float)(IB - QB) + fb;
            ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
            tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
            ev_in_cell = -1;
        }
        // the window's base moved by one along the event's axis
        const int q = evA ? 1 : (evB ? 2 : 0);
        df_sub(ah, al, q == 0 ? V.E1h[0] : (q == 1 ? V.E1h[1] : V.E1h[2]),
               q == 0 ? V.E1l[0] : (q == 1 ? V.E1l[1] : V.E1l[2]));
        df_sub(bh, bl, q == 0 ? V.E2h[0] : (q == 1 ? V.E2h[1] : V.E2h[2]),
               q == 0 ? V.E2l[0] : (q == 1 ? V.E2l[1] : V.E2l[2]));
        // the entering face: A: (x, N, y); B: (x, y, N); D: (N, x, y)
#pragma unroll
        for (int x = 0; x <= N; ++x)
#pragma unroll
            for (int y = 0; y <= N; ++y) visit(evD ? N : x, evA ? N : (evB ? y : x), evB ? N : y);
        if (!ADJ) {
            if (kahan) kahan_add(sum, comp, acc);
            else sum += acc;
            acc = 0.0f;
        }
        if (++ev_in_cell >= qr.cap) return false;
    }
    if (!ADJ) {
        if (kahan) kahan_add(sum, comp, acc);
        else sum += acc;
    }
    out = sum;
    return true;
}

// One thread per ray, 128-thread blocks of one view (the exact kernels'
// tiling); lookups read the table through L1/L2.  (Staging a view's table in
// shared memory, 202.5 KB for cubic, forces one 512-thread block per SM and
// measured slower.)
template <int N, bool ADJ>
__global__ void __launch_bounds__(128) k_table_pviews(DevGeom g, const float *__restrict__ cin, float *__restrict__ yout,
                                                      const float *__restrict__ yin, float *__restrict__ cout,
                                                      const float *__restrict__ T, int M, float inv_h, QuadRule qr,
                                                      int kahan, const __grid_constant__ ViewChunk vc)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const ViewConst &V = vc.v[blockIdx.z];
    const int k = V.view;
    if (iu >= g.nu || iv >= g.nv) return;
    const long long ray = ((long long)k * g.nv + iv) * g.nu + iu;
    float yr = 0.0f;
    if (ADJ) {
        yr = __ldg(yin + ray);
        if (yr == 0.0f) return;
    }
    RaySetup rs;
    float out = 0.0f;
    if (view_setup<N>(g, grid_of(g), k, iu, iv, rs)) {
        use_view_const(V, rs);
        const ViewPose &P = g.views[k];
        const double a = iu - 0.5 * (g.nu - 1), b = iv - 0.5 * (g.nv - 1);
        double al0 = 0.0, be0 = 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const double s = fma(b, P.dv[e], fma(a, P.du[e], P.dc[e])) - g.org[e];
            al0 = fma(s, P.e1[e], al0);
            be0 = fma(s, P.e2[e], be0);
        }
        const long long side = 2LL * M + 1;
        if (!table_march<N, ADJ>(rs, V, al0, be0, T + (long long)k * side * side, M, inv_h, cin, cout, yr, qr,
                                 kahan != 0, out))
            atomicOr(g.err, 1);
    }
    if (!ADJ) yout[ray] = out;
}

// ---------------------------------------------------------------- host side
namespace {
std::mutex g_table_mu;

template <int N>
spl_status build_table(spl_geometry *g, cudaStream_t st)
{
    TablePack &pk = g->table->pack[N];
    const int M = table_radius(N);
    const long long side = 2LL * M + 1, total = side * side * g->dev.n_views;
    float *T = nullptr;
    if (cudaMalloc(&T, (size_t)total * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        pk.state = -1;
        return fail(SPL_ERR_OOM, "footprint tables: cudaMalloc(%lld floats) failed", total);
    }
    k_table_build<N><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(g->dev, M, kTableStep, T, quad_rule(N));
    spl_status s = cuda_check(cudaGetLastError(), "table build");
    if (s == SPL_OK) s = cuda_check(cudaStreamSynchronize(st), "table build");
    if (s != SPL_OK) {
        cudaFree(T);
        pk.state = -1;
        return s;
    }
    pk.T = T;
    pk.M = M;
    pk.state = 1;
    return SPL_OK;
}

// The tables of `degree` exist (the projector allocates nothing: spl_prepare
// builds them).
spl_status table_ready(const spl_geometry *g, int degree)
{
    if (g->dev.kind != SPL_PARALLEL)
        return fail(SPL_ERR_UNSUPPORTED, "SPL_FP_TABLE needs a parallel-beam geometry (one footprint per view)");
    std::lock_guard<std::mutex> lock(g_table_mu);
    const int state = g->table ? g->table->pack[degree].state : 0;
    if (state == 1) return SPL_OK;
    if (state == -1) return fail(SPL_ERR_OOM, "footprint tables unavailable for this geometry and degree");
    return fail(SPL_ERR_STATE, "footprint tables of degree %d not built: call spl_prepare first", degree);
}

template <int N, bool ADJ>
spl_status table_launch(const spl_geometry *g, const spl_basis_desc *b, const float *cin, float *yout,
                        const float *yin, float *cout, cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    const TablePack &pk = g->table->pack[N];
    const QuadRule qr = quad_rule(N);
    const unsigned gx = (dg.nu + 15) / 16, gy = (dg.nv + 7) / 8;
    static thread_local ViewChunk ch;
    for (int s0 = 0; s0 < dg.n_views; s0 += kViewChunk) {
        const int n = dg.n_views - s0 < kViewChunk ? dg.n_views - s0 : kViewChunk;
        memcpy(ch.v, g->vconst + s0, (size_t)n * sizeof(ViewConst));
        k_table_pviews<N, ADJ><<<dim3(gx, gy, n), 128, 0, st>>>(
            dg, cin, yout, yin, cout, pk.T, pk.M, (float)(1.0 / kTableStep), qr, b->kahan, ch);
    }
    return cuda_check(cudaGetLastError(), "table projector launch");
}
}  // namespace

spl_status table_forward(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st)
{
    spl_status s = table_ready(g, b->degree);
    if (s != SPL_OK || g->dev.n_rays == 0) return s;
    switch (b->degree) {
    case 0: return table_launch<0, false>(g, b, c, y, nullptr, nullptr, st);
    case 1: return table_launch<1, false>(g, b, c, y, nullptr, nullptr, st);
    case 2: return table_launch<2, false>(g, b, c, y, nullptr, nullptr, st);
    default: return table_launch<3, false>(g, b, c, y, nullptr, nullptr, st);
    }
}

spl_status table_adjoint(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st)
{
    spl_status s = table_ready(g, b->degree);
    if (s != SPL_OK) return s;
    const long long nc = (long long)g->dev.n[0] * g->dev.n[1] * g->dev.n[2];
    s = cuda_check(cudaMemsetAsync(c, 0, nc * sizeof(float), st), "adjoint clear");
    if (s != SPL_OK || g->dev.n_rays == 0) return s;
    switch (b->degree) {
    case 0: return table_launch<0, true>(g, b, nullptr, nullptr, y, c, st);
    case 1: return table_launch<1, true>(g, b, nullptr, nullptr, y, c, st);
    case 2: return table_launch<2, true>(g, b, nullptr, nullptr, y, c, st);
    default: return table_launch<3, true>(g, b, nullptr, nullptr, y, c, st);
    }
}

spl_status table_build(spl_geometry *g, int degree, cudaStream_t st)
{
    if (g->dev.kind != SPL_PARALLEL)
        return fail(SPL_ERR_UNSUPPORTED, "SPL_FP_TABLE needs a parallel-beam geometry (one footprint per view)");
    std::lock_guard<std::mutex> lock(g_table_mu);
    if (!g->table) g->table = new TableSet();
    TablePack &pk = g->table->pack[degree];
    if (pk.state == 1) return SPL_OK;
    if (pk.state == -1) return fail(SPL_ERR_OOM, "footprint tables unavailable for this geometry and degree");
    switch (degree) {
    case 0: return build_table<0>(g, st);
    case 1: return build_table<1>(g, st);
    case 2: return build_table<2>(g, st);
    default: return build_table<3>(g, st);
    }
}

void table_free(TableSet *ts)
{
    if (!ts) return;
    for (int n = 0; n < 4; ++n)
        if (ts->pack[n].T) cudaFree(ts->pack[n].T);
    delete ts;
}

}  // namespace spl
