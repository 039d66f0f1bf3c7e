// spl_march.cuh -- device core of the B-spline x-ray transform (SplineSplat,
// arXiv 2511.11078): ray set-up, the dominant-axis cell march and the exact
// footprint engine shared by every kernel that walks a ray.
//
// Paper mapping
//   * Definition 2.1 (dominant axis d*): a ray is marched cell by cell along
//     d* = argmax |w_d| (ties: lowest index); every cell of d* that the ray's
//     reach covers is visited exactly once.
//   * Algorithm 2 / Algorithm 3: at each DDA step the bases of the slab
//     l_{d*} = k_{d*} within |l - k|_inf <= R are visited, minus those of the
//     two previous steps; over the ray, that is every basis whose support
//     the ray crosses, each once.  Here the same set is produced by an
//     (n+1)^3 register window of the bases whose support contains the
//     current point: a basis enters when the ray enters its support and is
//     flushed (c_l * P in the forward, y * P in the adjoint) exactly once
//     when it leaves, so no basis is visited twice and none is missed.
//   * Eq. 4 contribution Pphi(w, s - l): the integral along the ray of the
//     product of three 1-D B-splines.  Between consecutive knot-plane
//     crossings every factor of every window basis is one polynomial of
//     degree n, the product has degree 3n, and m = ceil((3n+1)/2)
//     Gauss-Legendre nodes integrate it exactly.  All (n+1)^3 window bases
//     share the nodes of a piece: each node costs 3 x (n+1) B-spline weights
//     and one (n+1)^3 outer product (cell_march, piece_march).
//
// Coordinates: index coordinates u = x - origin (bases at integers) are
// mirrored per axis so that the ray direction is componentwise >= 0
// (beta is even, so phi_l(x) = phi_{l'}(x') with l'_e = sign_e * l_e).
// The ray's transverse coordinates are carried as unevaluated float pairs
// (double-float) so that positions far from the origin keep ~1e-7 absolute
// accuracy without FP64 arithmetic in the hot loop.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace spl {

constexpr int kMaxNodes = 8;
// loop bound of the event loops: the knot crossings of one cell of the cell
// and piece marches (at most one per transverse axis, r <= 1), and the
// (n+1) d-pieces plus at most n+3 events per transverse axis of one slab of
// the pair enumeration, with margin
constexpr int kIterCap = 40;

struct QuadRule {
    float x[kMaxNodes];   // Gauss-Legendre nodes on [-1, 1], m = ceil((3n+1)/2) of them
    float w[kMaxNodes];   // weights
    float x1[kMaxNodes];  // the (n+1)-node rule: exact for degree 2n (flat rays, see cell_march)
    float w1[kMaxNodes];
    int cap;              // loop bound of the event loops (kIterCap)
};

// Direction-dependent part of the set-up (Definition 2.1 and the mirrored
// frame).  Parallel views share one per view (computed once on the host),
// other rays compute their own; the same function serves both so a ray gets
// the same values wherever it is set up.
struct DirSetup {
    int ax[3];          // axis index of (d, a, b): dominant axis, then the others by decreasing |w|
    int sg[3];          // mirror sign of (d, a, b)
    double r[2];        // |w_a|/|w_d|, |w_b|/|w_d| in [0, 1]
    double invr[2];     // 1 / r (0 when r == 0)
    float ra, rb, inv_ra, inv_rb, inv_wd;
    float rah, ral, rbh, rbl;  // r as double-float pairs
};

__host__ __device__ inline void dir_setup(const double (&w)[3], DirSetup &ds)
{
    double wp[3];
    int sg[3];
    for (int e = 0; e < 3; ++e) {
        sg[e] = (w[e] < 0.0) ? -1 : 1;
        wp[e] = w[e] < 0.0 ? -w[e] : w[e];
    }
    int d = 0;
    if (wp[1] > wp[d]) d = 1;
    if (wp[2] > wp[d]) d = 2;
    // transverse axes: a has the larger component (ties: lower index), so a
    // ray with one zero component always has r_b = 0
    int a = (d == 0) ? 1 : 0, b = (d == 2) ? 1 : 2;
    if (wp[b] > wp[a]) {
        const int tmp = a;
        a = b;
        b = tmp;
    }
    ds.ax[0] = d;
    ds.ax[1] = a;
    ds.ax[2] = b;
    ds.sg[0] = sg[d];
    ds.sg[1] = sg[a];
    ds.sg[2] = sg[b];
    const double iwd = 1.0 / wp[d];
    const double ra = wp[a] * iwd, rb = wp[b] * iwd;
    ds.r[0] = ra;
    ds.r[1] = rb;
    ds.invr[0] = ra > 0.0 ? 1.0 / ra : 0.0;
    ds.invr[1] = rb > 0.0 ? 1.0 / rb : 0.0;
    ds.rah = (float)ra;
    ds.ral = (float)(ra - (double)ds.rah);
    ds.rbh = (float)rb;
    ds.rbl = (float)(rb - (double)ds.rbh);
    ds.ra = ds.rah;
    ds.rb = ds.rbh;
    ds.inv_ra = ra > 0.0 ? (float)ds.invr[0] : INFINITY;
    ds.inv_rb = rb > 0.0 ? (float)ds.invr[1] : INFINITY;
    ds.inv_wd = (float)iwd;
}

// Constants of a parallel view that every ray of the view shares: the
// float part of its direction set-up, the mirrored strides and the grid
// bounds in its (d, a, b) frame.  The parallel-view kernels take them as a
// __grid_constant__ parameter indexed by blockIdx.z, so that they stay in
// the constant bank (uniform registers) instead of occupying per-thread
// registers next to the march window.
struct ViewConst {
    float ra, rb, inv_ra, inv_rb, inv_wd, rah, ral, rbh, rbl;
    int view;       // view index
    int S[3];       // signed linear strides of (d, a, b)
    int lo[3], hi[3];
    // footprint-table frame (e1, e2) of H_w in the mirrored (d, a, b) frame,
    // as double-float pairs: E1[q] = sg_q e1[ax_q]
    float E1h[3], E1l[3], E2h[3], E2l[3];
    // the scatter adjoint's copy of c: the layout whose contiguous axis is
    // b (0 x, 1 y, 2 z fast) and the strides of (d, a, b) in it
    int lay;
    int Sb[3];
};
constexpr int kViewChunk = 192;  // views per launch (26.25 KB of parameters)
struct ViewChunk {
    ViewConst v[kViewChunk];
};

__host__ __device__ inline void view_const(const DirSetup &ds, int view, const int (&n)[3], ViewConst &vc)
{
    const int stride[3] = {1, n[0], n[0] * n[1]};
    vc.ra = ds.ra;
    vc.rb = ds.rb;
    vc.inv_ra = ds.inv_ra;
    vc.inv_rb = ds.inv_rb;
    vc.inv_wd = ds.inv_wd;
    vc.rah = ds.rah;
    vc.ral = ds.ral;
    vc.rbh = ds.rbh;
    vc.rbl = ds.rbl;
    vc.view = view;
    // b-fast layouts: x fast [z][y][x], y fast [z][x][y], z fast [y][x][z]
    const int sb[3][3] = {{1, n[0], n[0] * n[1]}, {n[1], 1, n[0] * n[1]}, {n[2], n[0] * n[2], 1}};
    vc.lay = ds.ax[2];
    for (int q = 0; q < 3; ++q) {
        const int e = ds.ax[q];
        vc.S[q] = ds.sg[q] * stride[e];
        vc.Sb[q] = ds.sg[q] * sb[vc.lay][e];
        vc.lo[q] = ds.sg[q] > 0 ? 0 : -(n[e] - 1);
        vc.hi[q] = ds.sg[q] > 0 ? n[e] - 1 : 0;
    }
}

// the footprint-table frame of a parallel view in its mirrored frame
__host__ __device__ inline void view_const_frame(const DirSetup &ds, const double (&e1)[3], const double (&e2)[3],
                                                 ViewConst &vc)
{
    for (int q = 0; q < 3; ++q) {
        const double a = ds.sg[q] * e1[ds.ax[q]], b = ds.sg[q] * e2[ds.ax[q]];
        vc.E1h[q] = (float)a;
        vc.E1l[q] = (float)(a - (double)vc.E1h[q]);
        vc.E2h[q] = (float)b;
        vc.E2l[q] = (float)(b - (double)vc.E2h[q]);
    }
}

// Per-view pose in FP64 (one entry per view of a view geometry).
struct ViewPose {
    double src[3];       // parallel: unit ray direction; cone: source position
    double dc[3];        // detector centre
    double du[3], dv[3]; // detector axes (include the pixel pitch)
    double nrm[3];       // unit normal of the detector plane
    double ud[3], vd[3]; // dual axes: a = <P - dc, ud>, b = <P - dc, vd> for P on the plane
    DirSetup dir;        // parallel views: direction set-up shared by all rays of the view
    double e1[3], e2[3]; // parallel views: orthonormal frame of H_w of the footprint tables
};

struct DevGeom {
    int kind;            // SPL_RAYS / SPL_PARALLEL / SPL_CONE
    int n[3];            // nx, ny, nz
    double org[3];       // world position of coefficient (0,0,0)
    int n_views, nu, nv;
    long long n_rays;
    const ViewPose *views;
    const int *view_order;  // parallel views: the slice-separable group, the other flat views (r_b = 0), the rest
    int n_sep;              // views of the slice-separable group (view_order[0 .. n_sep))
    int n_flat;             // flat views, the group included (view_order[0 .. n_flat))
    const double *ray_w; // [n_rays][3] unit directions
    const double *ray_s; // [n_rays][3]
    // the caller's FP64 arrays as given: per view (direction or source,
    // detector centre, det_u, det_v), per ray (direction, point); the exact
    // pair count rebuilds each ray from them
    const double *raw;
    int *err;            // device error flag (bit 0: a loop bound was reached)
    size_t lay_cs;       // copy stride (floats) of the scatter adjoint's shifted layout copies
};

// ------------------------------------------------------------------ B-splines
// B_{n,i}(g) = beta^n(g + n - i - W), g in [0,1): weight of the i-th of the
// n+1 bases whose support contains a point, in power-basis coefficients.
template <int N> struct BSpl;
template <> struct BSpl<0> {
    __device__ static constexpr float c(int i, int k) { return 1.0f; }
};
template <> struct BSpl<1> {
    __device__ static constexpr float c(int i, int k)
    {
        return i == 0 ? (k == 0 ? 1.0f : -1.0f) : (k == 0 ? 0.0f : 1.0f);
    }
};
template <> struct BSpl<2> {
    __device__ static constexpr float c(int i, int k)
    {
        return i == 0   ? (k == 0 ? 0.5f : (k == 1 ? -1.0f : 0.5f))
               : i == 1 ? (k == 0 ? 0.5f : (k == 1 ? 1.0f : -1.0f))
                        : (k == 2 ? 0.5f : 0.0f);
    }
};
template <> struct BSpl<3> {
    __device__ static constexpr float c(int i, int k)
    {
        return i == 0   ? (k == 0 ? 1.0f / 6.0f : (k == 1 ? -0.5f : (k == 2 ? 0.5f : -1.0f / 6.0f)))
               : i == 1 ? (k == 0 ? 2.0f / 3.0f : (k == 1 ? 0.0f : (k == 2 ? -1.0f : 0.5f)))
               : i == 2 ? (k == 0 ? 1.0f / 6.0f : (k == 1 ? 0.5f : (k == 2 ? 0.5f : -0.5f)))
                        : (k == 3 ? 1.0f / 6.0f : 0.0f);
    }
};

template <int N> struct GL { static constexpr int M = (3 * N + 2) / 2 > 0 ? (3 * N + 2) / 2 : 1; };

// Weights of the N+1 bases whose support contains a point, with t = 1 - g.
// The outer weights vanish at an end of [0, 1] and are evaluated in factored
// form t^N/N!, g^N/N! (full relative accuracy near a support edge); the
// inner ones use the mirror symmetry B_{N,i}(g) = B_{N,N-i}(1 - g):
//   cubic:     w1 = 2/3 - g^2 (1 - g/2),  w2 = 2/3 - t^2 (1 - t/2)
//   quadratic: w1 = 1/2 + g t
// The mirror pairs (w_i, w_{N-i}) are evaluated as one packed FP32x2 pair
// (g, t): each component rounds like the scalar operation in the same
// order, so the weights are those of the scalar formulas in fewer
// instructions.
template <int N>
__device__ __forceinline__ void bweights(float g, float (&w)[N + 1])
{
    const float t = 1.0f - g;
    if constexpr (N == 0) {
        w[0] = 1.0f;
    } else if constexpr (N == 1) {
        w[0] = t;
        w[1] = g;
    } else if constexpr (N == 2) {
        // (0.5 g) g and (0.5 t) t
        const float2 gt = make_float2(g, t);
        const float2 e = __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), gt), gt);
        w[0] = e.y;
        w[1] = fmaf(g, t, 0.5f);
        w[2] = e.x;
    } else {
        const float2 gt = make_float2(g, t);
        const float2 sq = __fmul2_rn(gt, gt);                                           // g^2, t^2
        const float2 cu = __fmul2_rn(__fmul2_rn(sq, gt), make_float2(1.0f / 6.0f, 1.0f / 6.0f));  // w3, w0
        const float2 in = __ffma2_rn(make_float2(-0.5f, -0.5f), gt, make_float2(1.0f, 1.0f));
        const float2 md = __ffma2_rn(make_float2(-sq.x, -sq.y), in, make_float2(2.0f / 3.0f, 2.0f / 3.0f));  // w1, w2
        w[0] = cu.y;
        w[1] = md.x;
        w[2] = md.y;
        w[3] = cu.x;
    }
}

// ------------------------------------------------------------------ ray set-up
struct GridBox {
    int n[3];
    double org[3];
    int stride[3];   // linear-index strides of x, y, z
};

struct RaySetup {
    int ax[3];       // axis index of (d, a, b)
    int sg[3];       // mirror sign of (d, a, b)
    float ra, rb;    // |w_a|/|w_d|, |w_b|/|w_d|  in [0, 1]
    float inv_ra, inv_rb;
    float inv_wd;    // 1 / |w_d|
    int j0, j1;      // mirrored slab range (inclusive), reference slab j0
    int c0, c1;      // cell range of the cell march (inclusive), reference cell c0
    int lo[3], hi[3];  // mirrored grid bounds of (d, a, b)
    int S[3];        // signed linear strides of (d, a, b) in mirrored coordinates
    float Ah, Al, Bh, Bl;  // transverse coordinates at slab j0 (double-float)
    float Vah, Val, Vbh, Vbl;  // shifted transverse coordinates v = u + W at v_d = c0 (double-float)
    float rah, ral, rbh, rbl;
};

// Position-dependent part: slab and cell ranges of the ray and its
// transverse coordinates on the reference slab and cell.  Returns false when
// the ray meets no basis support of the grid.  FP64, a few dozen operations.
template <int N>
__device__ __forceinline__ bool pos_setup(const GridBox &gb, const DirSetup &ds, const double (&s)[3], RaySetup &rs)
{
    constexpr double W = 0.5 * (N + 1);
    double sp[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int e = ds.ax[q];
        rs.ax[q] = e;
        rs.sg[q] = ds.sg[q];
        rs.lo[q] = ds.sg[q] > 0 ? 0 : -(gb.n[e] - 1);
        rs.hi[q] = ds.sg[q] > 0 ? gb.n[e] - 1 : 0;
        rs.S[q] = ds.sg[q] * gb.stride[e];
        sp[q] = ds.sg[q] * (s[e] - gb.org[e]);
    }
    double jmin = rs.lo[0], jmax = rs.hi[0];
#pragma unroll
    for (int q = 1; q < 3; ++q) {
        const double r = ds.r[q - 1];
        if (r > 0.0) {
            const double m = W * (1.0 + r);
            jmin = fmax(jmin, fma(rs.lo[q] - m - sp[q], ds.invr[q - 1], sp[0]));
            jmax = fmin(jmax, fma(rs.hi[q] + m - sp[q], ds.invr[q - 1], sp[0]));
        } else if (!(sp[q] >= rs.lo[q] - W && sp[q] < rs.hi[q] + W)) {
            // constant transverse coordinate outside every support; the lower
            // end is inclusive for the half-open box of degree 0
            return false;
        }
    }
    // slab range: one slab of margin on both ends; extra slabs only add
    // empty windows
    rs.j0 = 0;
    rs.j1 = -1;
    if (jmax >= jmin - 1.0) {
        const double jl = fmax(floor(jmin) - 1.0, (double)rs.lo[0]);
        const double jh = fmin(ceil(jmax) + 1.0, (double)rs.hi[0]);
        if (jl <= jh) {
            rs.j0 = (int)jl;
            rs.j1 = (int)jh;
        }
    }
    // cell range (cell_march): with v = u + W, the grid's bases meet the
    // line where v_d is in (lo_d, hi_d + 2W) and each transverse v_e is in
    // (lo_e, hi_e + 2W); one cell of margin on both ends
    double vmin = rs.lo[0], vmax = rs.hi[0] + 2.0 * W;
#pragma unroll
    for (int q = 1; q < 3; ++q) {
        if (ds.r[q - 1] > 0.0) {
            vmin = fmax(vmin, fma(rs.lo[q] - W - sp[q], ds.invr[q - 1], sp[0] + W));
            vmax = fmin(vmax, fma(rs.hi[q] + W - sp[q], ds.invr[q - 1], sp[0] + W));
        }
    }
    rs.c0 = 0;
    rs.c1 = -1;
    if (vmax >= vmin - 1.0) {
        const double cl = fmax(floor(vmin) - 1.0, (double)rs.lo[0]);
        const double ch = fmin(floor(vmax) + 1.0, (double)(rs.hi[0] + N));
        if (cl <= ch) {
            rs.c0 = (int)cl;
            rs.c1 = (int)ch;
        }
    }
    if (rs.j0 > rs.j1 && rs.c0 > rs.c1) return false;
    const double A = fma(rs.j0 - sp[0], ds.r[0], sp[1]);
    const double B = fma(rs.j0 - sp[0], ds.r[1], sp[2]);
    rs.Ah = (float)A;
    rs.Al = (float)(A - (double)rs.Ah);
    rs.Bh = (float)B;
    rs.Bl = (float)(B - (double)rs.Bh);
    const double Va = fma(rs.c0 - W - sp[0], ds.r[0], sp[1]) + W;
    const double Vb = fma(rs.c0 - W - sp[0], ds.r[1], sp[2]) + W;
    rs.Vah = (float)Va;
    rs.Val = (float)(Va - (double)rs.Vah);
    rs.Vbh = (float)Vb;
    rs.Vbl = (float)(Vb - (double)rs.Vbh);
    rs.rah = ds.rah;
    rs.ral = ds.ral;
    rs.rbh = ds.rbh;
    rs.rbl = ds.rbl;
    rs.ra = ds.ra;
    rs.rb = ds.rb;
    rs.inv_ra = ds.inv_ra;
    rs.inv_rb = ds.inv_rb;
    rs.inv_wd = ds.inv_wd;
    return true;
}

// Ray in world coordinates -> slab-march set-up (both parts).  Shared by
// every kernel so that all of them enumerate the same pairs with the same
// footprint values.
template <int N>
__device__ __forceinline__ bool ray_setup(const GridBox &gb, const double (&s)[3], const double (&w)[3], RaySetup &rs)
{
    DirSetup ds;
    dir_setup(w, ds);
    return pos_setup<N>(gb, ds, s, rs);
}

// A + k r as integer + fraction in [0, 1], with A and r double-floats:
// TwoProduct (FMA) and TwoSum error-free transforms keep ~1e-7 absolute
// accuracy for |A| up to a few thousand.
__device__ __forceinline__ void df_coord(float Ah, float Al, float rh, float rl, int k, int &I, float &f)
{
    const float kf = (float)k;
    const float p = __fmul_rn(kf, rh);
    float pe = fmaf(kf, rh, -p);
    pe = fmaf(kf, rl, pe);
    const float s = __fadd_rn(Ah, p);
    const float bb = __fsub_rn(s, Ah);
    const float err = __fadd_rn(__fsub_rn(Ah, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float lo = __fadd_rn(__fadd_rn(err, pe), Al);
    const float fl = floorf(s);
    const float fr = __fadd_rn(__fsub_rn(s, fl), lo);
    const float adj = floorf(fr);
    I = (int)fl + (int)adj;
    f = __fsub_rn(fr, adj);
}

// ------------------------------------------------------------------ slab pairs
// Pairs of one slab j of a ray, without quadrature: every basis
// l' = (j, la, lb) whose support the ray crosses with positive length inside
// the slab is handed to sink.flush(j, la, lb, 1.0f) exactly once (the other
// bases of a window get 0).  A second DDA inside the slab runs over the knot
// planes of the transverse axes with a rolling (N+1) x (N+1) window of the
// bases whose support holds the current point; sink.relevant(a0, a1, b0, b1)
// says whether a window can reach the sink, sink.slab(IA, fa, IB, fb, N)
// receives the ray's transverse coordinates on the slab plane
// (A_j = IA + fa, B_j = IB + fb).  The learned-footprint projector enumerates
// its (ray, basis) pairs slab by slab with it, which bounds the pairs one
// round of a warp produces.  Returns false if the loop bound was reached.
template <int N, class Sink>
__device__ __forceinline__ bool slab_pairs(const RaySetup &rs, int j, const QuadRule &qr, Sink &sink)
{
    constexpr float W = 0.5f * (N + 1);
    int IA, IB;
    float fa, fb;
    df_coord(rs.Ah, rs.Al, rs.rah, rs.ral, j - rs.j0, IA, fa);
    df_coord(rs.Bh, rs.Bl, rs.rbh, rs.rbl, j - rs.j0, IB, fb);
    sink.slab(IA, fa, IB, fb, N);
    const float Ca = fa + W, Cb = fb + W;
    int qa = (int)floorf(fmaf(-W, rs.ra, Ca));
    int qb = (int)floorf(fmaf(-W, rs.rb, Cb));
    // r <= 1 moves a transverse coordinate by at most N+1 over the slab, so a
    // window shifts at most N+3 times per axis (one extra for a start that
    // rounds down); more is treated as a loop bound
    const int qa_lim = qa + N + 3, qb_lim = qb + N + 3;
    float na = rs.ra > 0.0f ? ((float)(qa + 1) - Ca) * rs.inv_ra : INFINITY;
    float nb = rs.rb > 0.0f ? ((float)(qb + 1) - Cb) * rs.inv_rb : INFINITY;
    float hit[N + 1][N + 1];  // 1 once the ray has crossed the basis' support
#pragma unroll
    for (int i = 0; i <= N; ++i)
#pragma unroll
        for (int k = 0; k <= N; ++k) hit[i][k] = 0.0f;
    float x0 = -W;
    int id = 0;  // d-piece: xi in [id - W, id + 1 - W)
#pragma unroll 1
    for (int it = 0; it < qr.cap; ++it) {
        const float nd = (float)(id + 1) - W;
        const float x1r = fminf(nd, fminf(na, nb));
        const int ev = (x1r == nd) ? 0 : ((x1r == na) ? 1 : 2);
        const float x1 = fmaxf(x1r, x0);
        const int la0 = IA + qa - N, lb0 = IB + qb - N;
        if (x1 > x0 && sink.relevant(la0, la0 + N, lb0, lb0 + N)) {
#pragma unroll
            for (int i = 0; i <= N; ++i)
#pragma unroll
                for (int k = 0; k <= N; ++k) hit[i][k] = 1.0f;
            sink.piece();
        }
        x0 = x1;
        if (ev == 0) {
            if (++id > N) {
#pragma unroll
                for (int i = 0; i <= N; ++i)
#pragma unroll
                    for (int k = 0; k <= N; ++k) sink.flush(j, la0 + i, lb0 + k, hit[i][k]);
                return true;
            }
        } else if (ev == 1) {
            // the lowest a-row leaves the ray's reach: flush it, shift
#pragma unroll
            for (int k = 0; k <= N; ++k) sink.flush(j, la0, lb0 + k, hit[0][k]);
#pragma unroll
            for (int i = 0; i < N; ++i)
#pragma unroll
                for (int k = 0; k <= N; ++k) hit[i][k] = hit[i + 1][k];
#pragma unroll
            for (int k = 0; k <= N; ++k) hit[N][k] = 0.0f;
            if (++qa > qa_lim) return false;
            na = ((float)(qa + 1) - Ca) * rs.inv_ra;
        } else {
            // the lowest b-column leaves
#pragma unroll
            for (int i = 0; i <= N; ++i) sink.flush(j, la0 + i, lb0, hit[i][0]);
#pragma unroll
            for (int i = 0; i <= N; ++i) {
#pragma unroll
                for (int k = 0; k < N; ++k) hit[i][k] = hit[i][k + 1];
                hit[i][N] = 0.0f;
            }
            if (++qb > qb_lim) return false;
            nb = ((float)(qb + 1) - Cb) * rs.inv_rb;
        }
    }
    return false;
}

// Region of bases a sink accepts, in the ray's mirrored (d, a, b)
// coordinates: lo[q] .. lo[q] + ext[q].
struct SinkBox {
    int lo0, lo1, lo2;
    unsigned ext0, ext1, ext2;
    __device__ __forceinline__ bool holds(int d, int a, int b) const
    {
        return (unsigned)(d - lo0) <= ext0 && (unsigned)(a - lo1) <= ext1 && (unsigned)(b - lo2) <= ext2;
    }
    __device__ __forceinline__ bool in0(int d) const { return (unsigned)(d - lo0) <= ext0; }
    __device__ __forceinline__ bool in1(int a) const { return (unsigned)(a - lo1) <= ext1; }
    __device__ __forceinline__ bool in2(int b) const { return (unsigned)(b - lo2) <= ext2; }
    // whether the cube [d0, d0+n] x [a0, a0+n] x [b0, b0+n] lies inside the region
    __device__ __forceinline__ bool cube_in(int d0, int a0, int b0, int n) const
    {
        return (unsigned)(d0 - lo0) + (unsigned)n <= ext0 && (unsigned)(d0 - lo0) <= ext0 &&
               (unsigned)(a0 - lo1) + (unsigned)n <= ext1 && (unsigned)(a0 - lo1) <= ext1 &&
               (unsigned)(b0 - lo2) + (unsigned)n <= ext2 && (unsigned)(b0 - lo2) <= ext2;
    }
    // whether the window [d0, d1] x [a0, a1] x [b0, b1] meets the region
    __device__ __forceinline__ bool meets(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return d1 >= lo0 && d0 <= lo0 + (int)ext0 && a1 >= lo1 && a0 <= lo1 + (int)ext1 && b1 >= lo2 &&
               b0 <= lo2 + (int)ext2;
    }
};

__device__ __forceinline__ SinkBox make_box(const int (&lo)[3], const int (&hi)[3])
{
    SinkBox b;
    b.lo0 = lo[0];
    b.lo1 = lo[1];
    b.lo2 = lo[2];
    b.ext0 = (unsigned)(hi[0] - lo[0]);
    b.ext1 = (unsigned)(hi[1] - lo[1]);
    b.ext2 = (unsigned)(hi[2] - lo[2]);
    return b;
}

// forward: sum of c_l * F_l along the ray, Kahan-compensated per cell
// compensated (Kahan) FP32 summation
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float v)
{
    const float yv = __fsub_rn(v, comp);
    const float t = __fadd_rn(sum, yv);
    comp = __fsub_rn(__fsub_rn(t, sum), yv);
    sum = t;
}

// Window update of one Gauss node, acc[d][i][k] += wd[d] wa[i] wb[k], with
// packed FP32x2 multiplies and FMAs two k at a time (__fmul2_rn,
// __ffma2_rn: each component rounds like the scalar operation, so the sums
// are those of the scalar loop, in half the instructions).
template <int N>
__device__ __forceinline__ void window_update(float (&acc)[N + 1][N + 1][N + 1], const float (&wd)[N + 1],
                                              const float (&wa)[N + 1], const float (&wb)[N + 1])
{
    constexpr int K2 = (N + 1) / 2;
    if constexpr (N == 3) {
        // pairs (3, 0) and (1, 2): the register pairs bweights<3> produces
        const float2 b30 = make_float2(wb[3], wb[0]), b12 = make_float2(wb[1], wb[2]);
#pragma unroll
        for (int i = 0; i <= N; ++i) {
            const float2 a2 = make_float2(wa[i], wa[i]);
            const float2 p30 = __fmul2_rn(a2, b30), p12 = __fmul2_rn(a2, b12);
#pragma unroll
            for (int d = 0; d <= N; ++d) {
                const float2 w2 = make_float2(wd[d], wd[d]);
                float2 u = make_float2(acc[d][i][3], acc[d][i][0]);
                u = __ffma2_rn(w2, p30, u);
                acc[d][i][3] = u.x;
                acc[d][i][0] = u.y;
                float2 v = make_float2(acc[d][i][1], acc[d][i][2]);
                v = __ffma2_rn(w2, p12, v);
                acc[d][i][1] = v.x;
                acc[d][i][2] = v.y;
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        float2 pk[K2 > 0 ? K2 : 1];
#pragma unroll
        for (int p = 0; p < K2; ++p)
            pk[p] = __fmul2_rn(make_float2(wa[i], wa[i]), make_float2(wb[2 * p], wb[2 * p + 1]));
        const float pl = ((N + 1) & 1) ? wa[i] * wb[N] : 0.0f;
#pragma unroll
        for (int d = 0; d <= N; ++d) {
            const float2 w2 = make_float2(wd[d], wd[d]);
#pragma unroll
            for (int p = 0; p < K2; ++p) {
                float2 a = make_float2(acc[d][i][2 * p], acc[d][i][2 * p + 1]);
                a = __ffma2_rn(w2, pk[p], a);
                acc[d][i][2 * p] = a.x;
                acc[d][i][2 * p + 1] = a.y;
            }
            if ((N + 1) & 1) acc[d][i][N] = fmaf(wd[d], pl, acc[d][i][N]);
        }
    }
}

// The flat form's update, acc[d][i][0] += wd[d] wa[i], two i at a time.
template <int N>
__device__ __forceinline__ void window_update_flat(float (&acc)[N + 1][N + 1][1], const float (&wd)[N + 1],
                                                   const float (&wa)[N + 1])
{
    constexpr int I2 = (N + 1) / 2;
#pragma unroll
    for (int d = 0; d <= N; ++d) {
        const float2 w2 = make_float2(wd[d], wd[d]);
#pragma unroll
        for (int p = 0; p < I2; ++p) {
            float2 a = make_float2(acc[d][2 * p][0], acc[d][2 * p + 1][0]);
            a = __ffma2_rn(w2, make_float2(wa[2 * p], wa[2 * p + 1]), a);
            acc[d][2 * p][0] = a.x;
            acc[d][2 * p + 1][0] = a.y;
        }
        if ((N + 1) & 1) acc[d][N][0] = fmaf(wd[d], wa[N], acc[d][N][0]);
    }
}

// f = sum_d wd[d] sum_i wa[i] sum_k wb[k] cw[d][i][k] (the direct march's
// node value), with packed FP32x2 FMAs over pairs of i.
template <int N>
__device__ __forceinline__ float window_contract(const float (&cw)[N + 1][N + 1][N + 1], const float (&wd)[N + 1],
                                                 const float (&wa)[N + 1], const float (&wb)[N + 1])
{
    constexpr int I2 = (N + 1) / 2;
    float f = 0.0f;
#pragma unroll
    for (int d = 0; d <= N; ++d) {
        float u = 0.0f;
        if constexpr (I2 > 0) {
            float2 u2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int p = 0; p < I2; ++p) {
                float2 t2 = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int k = 0; k <= N; ++k)
                    t2 = __ffma2_rn(make_float2(wb[k], wb[k]), make_float2(cw[d][2 * p][k], cw[d][2 * p + 1][k]), t2);
                u2 = __ffma2_rn(make_float2(wa[2 * p], wa[2 * p + 1]), t2, u2);
            }
            u = u2.x + u2.y;
        }
        if ((N + 1) & 1) {
            float tk = 0.0f;
#pragma unroll
            for (int k = 0; k <= N; ++k) tk = fmaf(wb[k], cw[d][N][k], tk);
            u = fmaf(wa[N], tk, u);
        }
        f = fmaf(wd[d], u, f);
    }
    return f;
}

// ------------------------------------------------------------------ cell march
// Cells along d*.  With v = u + W the bases of one axis sit at the integers
// and basis l covers v in (l, l + N + 1), so the N+1 bases whose support
// contains a point of cell [c, c+1) are l = c - N .. c, weighted by
// bweights(v - c).  The march walks the cells of a ray along d*.  Inside a
// cell the ray crosses at most one knot plane per transverse axis (r <= 1),
// so a cell splits into at most three pieces, and on each piece every factor
// of every live basis is one polynomial of degree N (product: degree 3N,
// GL<N>::M nodes).  An (N+1)^3 register window holds the live bases
// (offsets d, a, b) and all of them share each node's three weight sets:
// per node 3 (N+1) weights and (N+1)^3 FMAs.  When the ray crosses a
// transverse knot plane the bases behind it are flushed and the window
// shifts; at the end of a cell the lowest d-layer is flushed.  Each basis
// whose support the ray crosses is flushed exactly once, through
// sink.flush(l_d, l_a, l_b, F) with F = |w_d| Pphi(w, s - l) (the sink
// scales by 1/|w_d|).  Compared with a march slab by slab (Algorithm 2
// visits the bases of slab l_d = k_d at each step), which integrates every
// point of the ray once for each of the N+1 slabs whose d-support holds it,
// the node weights are evaluated once per point.
//
// Transverse positions: v_a at the start of cell c is a double-float
// (df_coord), exact to ~1e-7 anywhere on the ray.  The window's a-frame QA
// (it holds l_a = QA - N .. QA) only moves up; the a-crossings inside cell c
// are the integers in (QA, v_a(c+1)].  The window state at the start of a
// cell depends only on the cell, so a march over a sub-range of cells that
// starts before the first cell where a basis is live gives that basis the
// same value as the full march (the brick adjoint relies on it).
//
// FLAT (r_b = 0): the b-weights are constant along the ray; the window keeps
// the (N+1)^2 integrals over the d- and a-factors (degree 2N, N+1 nodes)
// and the flush multiplies them by the b-weights.
//
// Sink::plane (FLAT only): the sink takes G = F / w_b, one flush per
// (l_d, l_a), for the plane-matrix path of slice-separable views.
// Sink: relevant(d0, d1, a0, a1, b0, b1) says whether any basis of the
// window matters (pieces that reach none are not integrated); piece()
// counts an integrated piece; cell_end() closes a cell.  The per-cell event
// loop is bounded by qr.cap; reaching it (or a crossing count that r <= 1
// rules out) returns false.
template <int N, class Sink, bool FLAT>
__device__ __forceinline__ bool cell_march(const RaySetup &rs, int cf, int cl, const QuadRule &qr, Sink &sink)
{
    constexpr int NB = FLAT ? 1 : N + 1;
    constexpr int M = FLAT ? N + 1 : GL<N>::M;
    if (cf > cl) return true;
    float acc[N + 1][N + 1][NB];
#pragma unroll
    for (int d = 0; d <= N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k < NB; ++k) acc[d][i][k] = 0.0f;
    int IA, IB;
    float fa, fb;
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, cf - rs.c0, IA, fa);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, cf - rs.c0, IB, fb);
    int QA = IA, QB = IB;
    float wbf[N + 1];  // FLAT: the constant b-weights
    if constexpr (FLAT) bweights<N>(fb, wbf);
    // plane sinks (FLAT only) take the integrals over the d- and a-factors
    // themselves, one flush per (l_d, l_a) with l_b = 0
    constexpr bool PLANE = FLAT && Sink::plane;
    constexpr int KF = PLANE ? 1 : N + 1;
#define SPL_CELL_VAL(d, i, k) \
    (FLAT ? (PLANE ? acc[d][i][0] : acc[d][i][0] * wbf[k]) : acc[d][i][(FLAT ? 0 : k)])
#pragma unroll 1
    for (int c = cf; c <= cl; ++c) {
        int IAn, IBn = IB;
        float fan, fbn = fb;
        df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
        if constexpr (!FLAT) df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
        int na = IAn - QA, nb = IBn - QB;  // knot crossings inside the cell
        if (na > 2 || nb > 2) return false;
        float ga = (float)(IA - QA) + fa;  // v - frame at the cell start
        float gb = (float)(IB - QB) + fb;
        float ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
        float tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
        float t0 = 0.0f;
#pragma unroll 1
        for (int it = 0;; ++it) {
            if (it >= qr.cap) return false;
            const float t1 = fminf(fminf(ta, tb), 1.0f);
            if (t1 > t0 && sink.relevant(c - N, c, QA - N, QA, QB - N, QB)) {
                const float half = 0.5f * (t1 - t0), mid = 0.5f * (t0 + t1);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float t = fmaf(half, FLAT ? qr.x1[q] : qr.x[q], mid);
                    float wd[N + 1], wa[N + 1];
                    bweights<N>(t, wd);
                    bweights<N>(fmaf(rs.ra, t, ga), wa);
                    const float cw = half * (FLAT ? qr.w1[q] : qr.w[q]);
#pragma unroll
                    for (int d = 0; d <= N; ++d) wd[d] *= cw;
                    if constexpr (FLAT) {
                        window_update_flat<N>(acc, wd, wa);
                    } else {
                        float wb[N + 1];
                        bweights<N>(fmaf(rs.rb, t, gb), wb);
                        window_update<N>(acc, wd, wa, wb);
                    }
                }
                sink.piece();
            }
            t0 = fmaxf(t0, t1);
            if (ta <= tb && ta <= 1.0f) {
                // the lowest a-row leaves the ray's reach
#pragma unroll
                for (int d = 0; d <= N; ++d)
#pragma unroll
                    for (int k = 0; k < KF; ++k) sink.flush(c - N + d, QA - N, QB - N + k, SPL_CELL_VAL(d, 0, k));
#pragma unroll
                for (int d = 0; d <= N; ++d) {
#pragma unroll
                    for (int i = 0; i < N; ++i)
#pragma unroll
                        for (int k = 0; k < NB; ++k) acc[d][i][k] = acc[d][i + 1][k];
#pragma unroll
                    for (int k = 0; k < NB; ++k) acc[d][N][k] = 0.0f;
                }
                ++QA;
                ga -= 1.0f;
                ta = --na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
            } else if (tb <= 1.0f) {
                // the lowest b-column leaves (never for FLAT: nb == 0)
#pragma unroll
                for (int d = 0; d <= N; ++d)
#pragma unroll
                    for (int i = 0; i <= N; ++i) sink.flush(c - N + d, QA - N + i, QB - N, SPL_CELL_VAL(d, i, 0));
                if constexpr (!FLAT) {
#pragma unroll
                    for (int d = 0; d <= N; ++d)
#pragma unroll
                        for (int i = 0; i <= N; ++i) {
#pragma unroll
                            for (int k = 0; k < N; ++k) acc[d][i][(FLAT ? 0 : k)] = acc[d][i][(FLAT ? 0 : k + 1)];
                            acc[d][i][(FLAT ? 0 : N)] = 0.0f;
                        }
                }
                ++QB;
                gb -= 1.0f;
                tb = --nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
            } else {
                break;
            }
        }
        // end of the cell: the lowest d-layer leaves
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k < KF; ++k) sink.flush(c - N, QA - N + i, QB - N + k, SPL_CELL_VAL(0, i, k));
#pragma unroll
        for (int d = 0; d < N; ++d)
#pragma unroll
            for (int i = 0; i <= N; ++i)
#pragma unroll
                for (int k = 0; k < NB; ++k) acc[d][i][k] = acc[d + 1][i][k];
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k < NB; ++k) acc[N][i][k] = 0.0f;
        sink.cell_end();
        IA = IAn;
        fa = fan;
        IB = IBn;
        fb = fbn;
    }
    // what the window still holds (layers l_d = cl+1-N .. cl; the top one is
    // empty) is flushed once: bases outside the sink's region, or complete
    // ones when the cell range was clipped
#pragma unroll
    for (int d = 0; d < N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k < KF; ++k) sink.flush(cl + 1 - N + d, QA - N + i, QB - N + k, SPL_CELL_VAL(d, i, k));
    sink.cell_end();
#undef SPL_CELL_VAL
    return true;
}

// Piece march: the cell march of a general ray (r_b > 0) with one piece per
// loop iteration instead of one cell.  The cells, pieces, nodes, window and
// flushes are those of cell_march<N, Sink, false>; what differs is control
// flow.  The lanes of a warp hold rays whose cells split into different
// numbers of pieces (1 + a-crossings + b-crossings), so a loop over cells
// runs every cell as often as its most-split lane needs; here every lane
// integrates one piece per iteration whatever cell it is in, and the event
// that ends the piece (an a- or b-crossing, or the end of the cell) is
// handled without branches: the leaving face is picked with selects,
// flushed through sink.put(offset, in_region, F, slot) at offsets in the
// sink's layout (sink.S0..S2, sink.off, region sink.bx; slot in 0..N is the
// face entry's second index, so a sink may spread the face over N+1
// independent partial sums) -- or, when the whole window lies in the region
// and the sink has Sink::face, through one sink.put_face(base, SX, SY, F)
// of the face's (N+1)^2 values at base + x SX + y SY -- and the window shifted
// with selects along the event's axis.  Only the set-up of the next cell
// is a branch.  The Gauss weights carry the factor sink.wscale() (1, or the
// adjoint's y_r), so the values the sink receives already include it.
template <int N, class Sink>
__device__ __forceinline__ bool piece_march(const RaySetup &rs, int cf, int cl, const QuadRule &qr, Sink &sink)
{
    constexpr int M = GL<N>::M;
    if (cf > cl) return true;
    float acc[N + 1][N + 1][N + 1];
#pragma unroll
    for (int d = 0; d <= N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k <= N; ++k) acc[d][i][k] = 0.0f;
    int c = cf;
    int IA, IB, IAn, IBn;
    float fa, fb, fan, fbn;
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c - rs.c0, IA, fa);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c - rs.c0, IB, fb);
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
    int QA = IA, QB = IB;
    int na = IAn - QA, nb = IBn - QB;
    if (na > 2 || nb > 2) return false;
    float ga = fa, gb = fb;
    float ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
    float tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
    float t0 = 0.0f;
    int ev_in_cell = 0;
    bool ok = true;
#pragma unroll 1
    while (true) {
        const float t1 = fminf(fminf(ta, tb), 1.0f);
        if (t1 > t0 && sink.relevant(c - N, c, QA - N, QA, QB - N, QB)) {
            const float half = 0.5f * (t1 - t0), mid = 0.5f * (t0 + t1), hs = half * sink.wscale();
#pragma unroll
            for (int q = 0; q < M; ++q) {
                const float t = fmaf(half, qr.x[q], mid);
                float wd[N + 1], wa[N + 1], wb[N + 1];
                bweights<N>(t, wd);
                bweights<N>(fmaf(rs.ra, t, ga), wa);
                bweights<N>(fmaf(rs.rb, t, gb), wb);
                const float cw = hs * qr.w[q];
#pragma unroll
                for (int d = 0; d <= N; ++d) wd[d] *= cw;
                window_update<N>(acc, wd, wa, wb);
            }
            sink.piece();
        }
        t0 = fmaxf(t0, t1);
        const bool evA = ta <= tb && ta <= 1.0f;
        const bool evB = !evA && tb <= 1.0f;
        const bool evD = !evA && !evB;
        // the face that leaves: A: (d = x, i = 0, k = y); B: (d = x, i = y,
        // k = 0); D: (d = 0, i = x, k = y)
        {
            const int bd = c - N, ba = QA - N, bb = QB - N;
            const unsigned base = sink.off + (unsigned)bd * (unsigned)sink.S0 + (unsigned)ba * (unsigned)sink.S1 +
                                  (unsigned)bb * (unsigned)sink.S2;
            const unsigned SX = (unsigned)(evD ? sink.S1 : sink.S0), SY = (unsigned)(evB ? sink.S1 : sink.S2);
            if (sink.bx.cube_in(bd, ba, bb, N)) {
                // the whole window lies in the region (most pieces): every
                // face entry is in, no per-entry tests
                if constexpr (Sink::face) {
                    float fv[N + 1][N + 1];
#pragma unroll
                    for (int x = 0; x <= N; ++x)
#pragma unroll
                        for (int y = 0; y <= N; ++y)
                            fv[x][y] = evA ? acc[x][0][y] : (evB ? acc[x][y][0] : acc[0][x][y]);
                    sink.template put_face<N>(base, SX, SY, fv);
                } else {
#pragma unroll
                    for (int x = 0; x <= N; ++x)
#pragma unroll
                        for (int y = 0; y <= N; ++y) {
                            const float v = evA ? acc[x][0][y] : (evB ? acc[x][y][0] : acc[0][x][y]);
                            sink.put(base + (unsigned)x * SX + (unsigned)y * SY, true, v, y);
                        }
                }
            } else {
                const bool vf = evA ? sink.bx.in1(ba) : (evB ? sink.bx.in2(bb) : sink.bx.in0(bd));
                bool vx[N + 1], vy[N + 1];
#pragma unroll
                for (int x = 0; x <= N; ++x) {
                    vx[x] = vf && (evD ? sink.bx.in1(ba + x) : sink.bx.in0(bd + x));
                    vy[x] = evB ? sink.bx.in1(ba + x) : sink.bx.in2(bb + x);
                }
#pragma unroll
                for (int x = 0; x <= N; ++x)
#pragma unroll
                    for (int y = 0; y <= N; ++y) {
                        const float v = evA ? acc[x][0][y] : (evB ? acc[x][y][0] : acc[0][x][y]);
                        sink.put(base + (unsigned)x * SX + (unsigned)y * SY, vx[x] && vy[y], v, y);
                    }
            }
        }
        // shift along the event's axis (in place: reads only higher indices)
#pragma unroll
        for (int d = 0; d <= N; ++d)
#pragma unroll
            for (int i = 0; i <= N; ++i)
#pragma unroll
                for (int k = 0; k <= N; ++k) {
                    const float nd = d < N ? acc[(d < N ? d + 1 : d)][i][k] : 0.0f;
                    const float na_ = i < N ? acc[d][(i < N ? i + 1 : i)][k] : 0.0f;
                    const float nb_ = k < N ? acc[d][i][(k < N ? k + 1 : k)] : 0.0f;
                    acc[d][i][k] = evD ? nd : (evA ? na_ : nb_);
                }
        if (evA) {
            ++QA;
            ga -= 1.0f;
            ta = --na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
        } else if (evB) {
            ++QB;
            gb -= 1.0f;
            tb = --nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
        } else {
            sink.cell_end();
            if (++c > cl) break;
            IA = IAn;
            fa = fan;
            IB = IBn;
            fb = fbn;
            df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
            df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
            na = IAn - QA;
            nb = IBn - QB;
            if (na > 2 || nb > 2) {
                ok = false;
                break;
            }
            ga = (float)(IA - QA) + fa;
            gb = (float)(IB - QB) + fb;
            ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
            tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
            t0 = 0.0f;
            ev_in_cell = -1;
        }
        if (++ev_in_cell >= qr.cap) {
            ok = false;
            break;
        }
    }
    if (!ok) return false;
    // what the window still holds (layers l_d = cl+1-N .. cl) is flushed once
#pragma unroll
    for (int d = 0; d < N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k <= N; ++k) {
                const int ld = cl + 1 - N + d, la = QA - N + i, lb = QB - N + k;
                const unsigned off = sink.off + (unsigned)ld * (unsigned)sink.S0 + (unsigned)la * (unsigned)sink.S1 +
                                     (unsigned)lb * (unsigned)sink.S2;
                sink.put(off, sink.bx.in0(ld) && sink.bx.in1(la) && sink.bx.in2(lb), acc[d][i][k], k);
            }
    sink.cell_end();
    return true;
}

// Direct march (the forward only): the line integral of f itself along the
// ray, f(x) = sum_l c_l phi_l(x), over the same cells, pieces and Gauss
// nodes as the piece march.  The window holds the coefficients of the live
// bases (zero outside the grid) instead of their footprint accumulators:
// each node contracts them with its three weight sets,
//   f = sum_d wd_d sum_i wa_i sum_k wb_k c[d][i][k],
// and an event shifts the window and loads the entering face (16 gathers)
// instead of flushing the leaving one.  The matrix is the same as the
// footprint form's; only the FP32 rounding differs.
// CX: coefficient array; S0..S2, bx: mirrored strides and grid bounds.
template <int N>
__device__ __forceinline__ bool direct_march(const RaySetup &rs, const float *__restrict__ CX, int S0, int S1, int S2,
                                             const SinkBox &bx, const QuadRule &qr, bool kahan, float &out)
{
    constexpr int M = GL<N>::M;
    out = 0.0f;
    const int cf = rs.c0, cl = rs.c1;
    if (cf > cl) return true;
    int c = cf;
    int IA, IB, IAn, IBn;
    float fa, fb, fan, fbn;
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c - rs.c0, IA, fa);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c - rs.c0, IB, fb);
    df_coord(rs.Vah, rs.Val, rs.rah, rs.ral, c + 1 - rs.c0, IAn, fan);
    df_coord(rs.Vbh, rs.Vbl, rs.rbh, rs.rbl, c + 1 - rs.c0, IBn, fbn);
    int QA = IA, QB = IB;
    // the window of cell c: l = (c - N + d, QA - N + i, QB - N + k)
    float cw[N + 1][N + 1][N + 1];
#pragma unroll
    for (int d = 0; d <= N; ++d)
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
            for (int k = 0; k <= N; ++k) {
                const int ld = c - N + d, la = QA - N + i, lb = QB - N + k;
                const unsigned o = (unsigned)ld * (unsigned)S0 + (unsigned)la * (unsigned)S1 + (unsigned)lb * (unsigned)S2;
                cw[d][i][k] = (bx.in0(ld) && bx.in1(la) && bx.in2(lb)) ? __ldg(CX + o) : 0.0f;
            }
    int na = IAn - QA, nb = IBn - QB;
    if (na > 2 || nb > 2) return false;
    float ga = fa, gb = fb;
    float ta = na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
    float tb = nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
    float t0 = 0.0f, cell = 0.0f, sum = 0.0f, comp = 0.0f;
    int ev_in_cell = 0;
#pragma unroll 1
    while (true) {
        const float t1 = fminf(fminf(ta, tb), 1.0f);
        if (t1 > t0 && bx.meets(c - N, c, QA - N, QA, QB - N, QB)) {
            const float half = 0.5f * (t1 - t0), mid = 0.5f * (t0 + t1);
            float piece = 0.0f;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                const float t = fmaf(half, qr.x[q], mid);
                float wd[N + 1], wa[N + 1], wb[N + 1];
                bweights<N>(t, wd);
                bweights<N>(fmaf(rs.ra, t, ga), wa);
                bweights<N>(fmaf(rs.rb, t, gb), wb);
                const float f = window_contract<N>(cw, wd, wa, wb);
                piece = fmaf(qr.w[q], f, piece);
            }
            cell = fmaf(half, piece, cell);
        }
        t0 = fmaxf(t0, t1);
        const bool evA = ta <= tb && ta <= 1.0f;
        const bool evB = !evA && tb <= 1.0f;
        const bool evD = !evA && !evB;
        // the entering face after the shift: A: (d = x, i = N, k = y);
        // B: (d = x, i = y, k = N); D: (d = N, i = x, k = y)
        float L[N + 1][N + 1];
        {
            const int bd = evD ? c + 1 : c - N, ba = evA ? QA + 1 : QA - N, bb = evB ? QB + 1 : QB - N;
            const unsigned base = (unsigned)bd * (unsigned)S0 + (unsigned)ba * (unsigned)S1 + (unsigned)bb * (unsigned)S2;
            const unsigned SX = (unsigned)(evD ? S1 : S0), SY = (unsigned)(evB ? S1 : S2);
            const bool vf = evA ? bx.in1(ba) : (evB ? bx.in2(bb) : bx.in0(bd));
            bool vx[N + 1], vy[N + 1];
#pragma unroll
            for (int x = 0; x <= N; ++x) {
                vx[x] = vf && (evD ? bx.in1(ba + x) : bx.in0(bd + x));
                vy[x] = evB ? bx.in1(ba + x) : bx.in2(bb + x);
            }
            const bool load = !(evD && c + 1 > cl);  // no cell after the last one
#pragma unroll
            for (int x = 0; x <= N; ++x)
#pragma unroll
                for (int y = 0; y <= N; ++y)
                    L[x][y] = (load && vx[x] && vy[y]) ? __ldg(CX + (base + (unsigned)x * SX + (unsigned)y * SY)) : 0.0f;
        }
#pragma unroll
        for (int d = 0; d <= N; ++d)
#pragma unroll
            for (int i = 0; i <= N; ++i)
#pragma unroll
                for (int k = 0; k <= N; ++k) {
                    const float nd = d < N ? cw[(d < N ? d + 1 : d)][i][k] : L[i][k];
                    const float na_ = i < N ? cw[d][(i < N ? i + 1 : i)][k] : L[d][k];
                    const float nb_ = k < N ? cw[d][i][(k < N ? k + 1 : k)] : L[d][i];
                    cw[d][i][k] = evD ? nd : (evA ? na_ : nb_);
                }
        if (evA) {
            ++QA;
            ga -= 1.0f;
            ta = --na > 0 ? fminf((1.0f - ga) * rs.inv_ra, 1.0f) : 2.0f;
        } else if (evB) {
            ++QB;
            gb -= 1.0f;
            tb = --nb > 0 ? fminf((1.0f - gb) * rs.inv_rb, 1.0f) : 2.0f;
        } else {
            const float v = cell * rs.inv_wd;
            cell = 0.0f;
            if (kahan) kahan_add(sum, comp, v);
            else sum += v;
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
            t0 = 0.0f;
            ev_in_cell = -1;
        }
        if (++ev_in_cell >= qr.cap) return false;
    }
    out = sum;
    return true;
}

// March over cells [cf, cl] with the form the ray needs: the flat cell march
// when the ray has a zero transverse component (r_b = 0), the piece march
// otherwise.  Every exact-footprint kernel goes through here, so a ray gets
// the same footprint values in the forward, the adjoint, the pair count and
// the footprint evaluator.
template <int N, class Sink>
__device__ __forceinline__ bool march(const RaySetup &rs, int cf, int cl, const QuadRule &qr, Sink &sink)
{
    if (rs.rb == 0.0f) return cell_march<N, Sink, true>(rs, cf, cl, qr, sink);
    return piece_march<N, Sink>(rs, cf, cl, qr, sink);
}

// pixel of this thread in a view kernel: a 128-thread block covers a 16 x 8
// detector tile, a warp an 8 x 4 sub-tile
__device__ __forceinline__ void tile_pixel(int &iu, int &iv)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    iu = blockIdx.x * 16 + (wid & 1) * 8 + (lane & 7);
    iv = blockIdx.y * 8 + (wid >> 1) * 4 + (lane >> 3);
}

// Rays of a parallel view: the view's constants replace the set-up's
// per-thread copies of the same values, so the march reads them from the
// kernel parameter (uniform across the block).
__device__ __forceinline__ void use_view_const(const ViewConst &V, RaySetup &rs)
{
    rs.ra = V.ra;
    rs.rb = V.rb;
    rs.inv_ra = V.inv_ra;
    rs.inv_rb = V.inv_rb;
    rs.inv_wd = V.inv_wd;
    rs.rah = V.rah;
    rs.ral = V.ral;
    rs.rbh = V.rbh;
    rs.rbl = V.rbl;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        rs.S[q] = V.S[q];
        rs.lo[q] = V.lo[q];
        rs.hi[q] = V.hi[q];
    }
}

// ------------------------------------------------------------------ rays of a geometry
__device__ __forceinline__ void view_ray(const DevGeom &g, int k, int iu, int iv, double (&s)[3], double (&w)[3])
{
    const ViewPose &P = g.views[k];
    const double a = iu - 0.5 * (g.nu - 1), b = iv - 0.5 * (g.nv - 1);
    double q[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) q[e] = fma(b, P.dv[e], fma(a, P.du[e], P.dc[e]));
    if (g.kind == 1) {
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            s[e] = q[e];
            w[e] = P.src[e];
        }
    } else {
        double dd[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) dd[e] = q[e] - P.src[e];
        const double nrm = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            s[e] = P.src[e];
            w[e] = dd[e] / nrm;
        }
    }
}

// Set up pixel (iu, iv) of view k.  Parallel views take the per-view
// direction set-up and only compute the pixel position; cone rays set up
// their own direction.
template <int N>
__device__ __forceinline__ bool view_setup(const DevGeom &g, const GridBox &gb, int k, int iu, int iv, RaySetup &rs)
{
    double s[3], w[3];
    if (g.kind == 1) {
        const ViewPose &P = g.views[k];
        const double a = iu - 0.5 * (g.nu - 1), b = iv - 0.5 * (g.nv - 1);
#pragma unroll
        for (int e = 0; e < 3; ++e) s[e] = fma(b, P.dv[e], fma(a, P.du[e], P.dc[e]));
        return pos_setup<N>(gb, P.dir, s, rs);
    }
    view_ray(g, k, iu, iv, s, w);
    return ray_setup<N>(gb, s, w, rs);
}

__device__ __forceinline__ void explicit_ray(const DevGeom &g, long long r, double (&s)[3], double (&w)[3])
{
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        s[e] = g.ray_s[3 * r + e];
        w[e] = g.ray_w[3 * r + e];
    }
}

__device__ __forceinline__ GridBox grid_of(const DevGeom &g)
{
    GridBox gb;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        gb.n[e] = g.n[e];
        gb.org[e] = g.org[e];
    }
    gb.stride[0] = 1;
    gb.stride[1] = g.n[0];
    gb.stride[2] = g.n[0] * g.n[1];
    return gb;
}


}  // namespace spl
