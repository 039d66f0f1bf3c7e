// plane.cu -- slice-separable parallel views: the plane-matrix path.
//
// A parallel view whose direction has a zero b component and whose
// detector rows run along b has flat rays (the b coordinate is constant
// along each ray, z_v for detector row v), and the tensor-product footprint
// factors exactly (Eq. 4 with phi = beta x beta x beta):
//   Pphi(w, s - l) = G(u; l_p, l_q) * beta^n(z_v - l_b),
//   G(u; l_p, l_q) = int beta^n(x_p(t) - l_p) beta^n(x_q(t) - l_q) dt,
// where the integral runs along the ray's path in the (p, q) plane, which
// depends on the detector column u only.  The forward projection of such a
// view is therefore
//   y(u, v) = sum_(l_p, l_q) G(u; l_p, l_q) S(l_p, l_q; v),
//   S(l_p, l_q; v) = sum_(l_b) beta^n(z_v - l_b) c_l,
// and its adjoint
//   c_l += sum_v beta^n(z_v - l_b) T(l_p, l_q; v),
//   T(l_p, l_q; v) = sum_u G(u; l_p, l_q) y(u, v).
// G is the flat cell march of the column's ray with the b factor left out
// (the same march, rule and values every flat ray of the 3-D path uses).
// For a group of views that share b, the b coordinate of the detector centre
// and the b step of det_v, the rows of G (one per view and column) are
// stored once per degree in CSR form together with the transpose (CSC),
// so that the forward gathers rows and the adjoint gathers columns: no
// atomics, and the two use the same G values (the adjoint is matched to
// the forward exactly, up to FP32 summation order).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "spl_host.h"

namespace spl {

// ---------------------------------------------------------------- plane rows
// Sink of the flat cell march that records the plane footprint of every
// in-grid (l_d, l_a) basis: column index sd * l_d + sa * l_a (mirrored
// indices times the signed column strides), value G / |w_d|.
struct PlaneSink {
    static constexpr bool plane = true;
    int lo_d, hi_d, lo_a, hi_a;  // mirrored in-plane bounds
    int sd, sa;                  // signed column strides of d and a
    float scale;                 // 1 / |w_d|
    int *col;                    // fill mode: output arrays (NULL: count only)
    float *val;
    long long cap;
    long long n;
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ void cell_end() {}
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int, int) const
    {
        return d1 >= lo_d && d0 <= hi_d && a1 >= lo_a && a0 <= hi_a;
    }
    __device__ __forceinline__ void flush(int ld, int la, int, float v)
    {
        if (v != 0.0f && ld >= lo_d && ld <= hi_d && la >= lo_a && la <= hi_a) {
            if (col && n < cap) {
                col[n] = sd * ld + sa * la;
                val[n] = v * scale;
            }
            ++n;
        }
    }
};

struct PlaneArgs {
    int n_p, b;                  // col = i_q * n_p + i_p; separable axis
    int nu;
    long long rows;
};

// One thread per plane row r = (group view gi, column u): set up the ray of
// pixel (u, any row) with its b coordinate moved to the middle of the grid
// (flat rays: the plane path does not depend on it) and march its cells.
// COUNT: row lengths into row_ptr[r]; FILL: entries at row_ptr[r].
template <int N, bool FILL>
__global__ void __launch_bounds__(128) k_plane_rows(DevGeom g, PlaneArgs pa, long long *row_ptr, int *row_col,
                                                    float *row_val, QuadRule qr)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= pa.rows) return;
    const int gi = (int)(r / pa.nu), u = (int)(r % pa.nu);
    const ViewPose &P = g.views[g.view_order[gi]];
    const double a = u - 0.5 * (g.nu - 1);
    double s[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) s[e] = fma(a, P.du[e], P.dc[e]);
    s[pa.b] = g.org[pa.b] + 0.5 * (g.n[pa.b] - 1);
    const GridBox gb = grid_of(g);
    RaySetup rs;
    PlaneSink sk;
    sk.n = 0;
    sk.col = nullptr;
    sk.val = nullptr;
    sk.cap = 0;
    if (pos_setup<N>(gb, P.dir, s, rs)) {
        sk.lo_d = rs.lo[0];
        sk.hi_d = rs.hi[0];
        sk.lo_a = rs.lo[1];
        sk.hi_a = rs.hi[1];
        sk.sd = rs.sg[0] * (rs.ax[0] == (pa.b == 0 ? 1 : 0) ? 1 : pa.n_p);
        sk.sa = rs.sg[1] * (rs.ax[1] == (pa.b == 0 ? 1 : 0) ? 1 : pa.n_p);
        sk.scale = rs.inv_wd;
        if (FILL) {
            const long long e0 = row_ptr[r];
            sk.col = row_col + e0;
            sk.val = row_val + e0;
            sk.cap = row_ptr[r + 1] - e0;
        }
        if (!cell_march<N, PlaneSink, true>(rs, rs.c0, rs.c1, qr, sk)) atomicOr(g.err, 1);
    }
    if (!FILL) row_ptr[r] = sk.n;
    else if (sk.n != sk.cap) atomicOr(g.err, 2);
}

// Exclusive scan of a[0..n) in place, a[n] = total (one block).
__global__ void __launch_bounds__(1024) k_scan(long long *a, long long n)
{
    __shared__ long long part[1024];
    __shared__ long long total;
    const int t = threadIdx.x;
    const long long per = (n + 1023) / 1024;
    const long long lo = t * per, hi = lo + per < n ? lo + per : n;
    long long s = 0;
    for (long long i = lo; i < hi; ++i) s += a[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        for (int i = 0; i < 1024; ++i) {
            const long long v = part[i];
            part[i] = run;
            run += v;
        }
        total = run;
    }
    __syncthreads();
    long long run = part[t];
    for (long long i = lo; i < hi; ++i) {
        const long long v = a[i];
        a[i] = run;
        run += v;
    }
    if (t == 0) a[n] = total;
}

// column counts (into col_ptr[col]) and the transpose fill
__global__ void __launch_bounds__(128) k_plane_colcount(long long rows, const long long *row_ptr, const int *row_col,
                                                        long long *col_cnt)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (long long e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
        atomicAdd((unsigned long long *)(col_cnt + row_col[e]), 1ull);
}

__global__ void __launch_bounds__(128) k_plane_colfill(long long rows, const long long *row_ptr, const int *row_col,
                                                       const float *row_val, long long *cursor, int *col_row,
                                                       float *col_val)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    for (long long e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        const long long pos = (long long)atomicAdd((unsigned long long *)(cursor + row_col[e]), 1ull);
        col_row[pos] = (int)r;
        col_val[pos] = row_val[e];
    }
}

// ---------------------------------------------------------------- per-call kernels
struct PlaneCall {
    int n_p, n_q, n_b;           // grid sizes of p, q, b
    long long st_p, st_q, st_b;  // linear strides of p, q, b in c
    long long ncol, rows;
    int nu, nv;
};

// S[col][v] = sum_i wz[v][i] c(col, lb0[v] + i)
template <int N>
__global__ void __launch_bounds__(256) k_plane_zres(PlaneCall pc, const float *__restrict__ c, const int *lb0,
                                                    const float *wz, float *__restrict__ S)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pc.ncol * pc.nv) return;
    const int v = (int)(idx % pc.nv);
    const long long col = idx / pc.nv;
    const long long ip = col % pc.n_p, iq = col / pc.n_p;
    const float *cc = c + ip * pc.st_p + iq * pc.st_q;
    const int l0 = lb0[v];
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i <= N; ++i) {
        const int lb = l0 + i;
        if (lb >= 0 && lb < pc.n_b) s = fmaf(wz[v * (N + 1) + i], __ldg(cc + lb * pc.st_b), s);
    }
    S[idx] = s;
}

// Warp-per-row sparse gather: out[row][v] = sum_e val[e] * in[idx[e]][v]
// (rows of the forward, columns of the adjoint).  Lanes cover v; each chunk
// of 32 entries is loaded once and broadcast by shuffles.  KAHAN: the chunk
// partials are added with compensation.
constexpr int kPlaneWarps = 8;
constexpr int kPlaneMV = 8;  // v per lane per pass (256 v per pass)

template <bool KAHAN, bool TO_Y>
__global__ void __launch_bounds__(32 * kPlaneWarps) k_plane_gather(long long nrow, const long long *__restrict__ ptr,
                                                                   const int *__restrict__ idx,
                                                                   const float *__restrict__ val,
                                                                   const float *__restrict__ in, float *__restrict__ out,
                                                                   int nv, int nu, const int *view_order)
{
    const long long r = (long long)blockIdx.x * kPlaneWarps + (threadIdx.x >> 5);
    if (r >= nrow) return;
    const int lane = threadIdx.x & 31;
    const long long e0 = ptr[r], e1 = ptr[r + 1];
    for (int vb = 0; vb < nv; vb += 32 * kPlaneMV) {
        float acc[kPlaneMV], sum[kPlaneMV], comp[kPlaneMV];
#pragma unroll
        for (int m = 0; m < kPlaneMV; ++m) acc[m] = sum[m] = comp[m] = 0.0f;
        for (long long e = e0; e < e1; e += 32) {
            const int n = (int)(e1 - e < 32 ? e1 - e : 32);
            int mi = 0;
            float mv = 0.0f;
            if (lane < n) {
                mi = idx[e + lane];
                mv = val[e + lane];
            }
            for (int j = 0; j < n; ++j) {
                const long long ij = __shfl_sync(0xffffffffu, mi, j);
                const float gj = __shfl_sync(0xffffffffu, mv, j);
                const float *src = in + ij * nv + vb + lane;
#pragma unroll
                for (int m = 0; m < kPlaneMV; ++m)
                    if (vb + lane + 32 * m < nv) acc[m] = fmaf(gj, __ldg(src + 32 * m), acc[m]);
            }
            if (KAHAN) {
#pragma unroll
                for (int m = 0; m < kPlaneMV; ++m) {
                    kahan_add(sum[m], comp[m], acc[m]);
                    acc[m] = 0.0f;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < kPlaneMV; ++m) {
            const int v = vb + lane + 32 * m;
            if (v >= nv) continue;
            const float o = KAHAN ? sum[m] : acc[m];
            if (TO_Y) {
                const int gi = (int)(r / nu), u = (int)(r % nu);
                out[((long long)view_order[gi] * nv + v) * nu + u] = o;
            } else {
                out[r * nv + v] = o;
            }
        }
    }
}

// yt[gi*nu + u][v] = y[view_order[gi]][v][u]: 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) k_plane_ytrans(const float *__restrict__ y, float *__restrict__ yt,
                                                      const int *view_order, int nu, int nv)
{
    __shared__ float tile[32][33];
    const int gi = blockIdx.z;
    const int u0 = blockIdx.x * 32, v0 = blockIdx.y * 32;
    const long long k = view_order[gi];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int j = ty; j < 32; j += 8) {
        const int u = u0 + tx, v = v0 + j;
        tile[j][tx] = (u < nu && v < nv) ? __ldg(y + (k * nv + v) * nu + u) : 0.0f;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int u = u0 + j, v = v0 + tx;
        if (u < nu && v < nv) yt[((long long)gi * nu + u) * nv + v] = tile[tx][j];
    }
}

// c(col, lb) = sum_(v in vr[lb]) wz[v][lb - lb0[v]] * T[col][v]  (every
// coefficient written; ADD: added to what c holds)
template <int N, bool ADD>
__global__ void __launch_bounds__(256) k_plane_zadj(PlaneCall pc, const float *__restrict__ T, const int *lb0,
                                                    const float *wz, const int *vr, float *__restrict__ c)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= pc.ncol * pc.n_b) return;
    const long long col = idx % pc.ncol;
    const int lb = (int)(idx / pc.ncol);
    const long long ip = col % pc.n_p, iq = col / pc.n_p;
    float s = 0.0f;
    const int v0 = vr[2 * lb], v1 = vr[2 * lb + 1];
    for (int v = v0; v <= v1; ++v) {
        const int i = lb - lb0[v];
        if (i >= 0 && i <= N) s = fmaf(wz[v * (N + 1) + i], __ldg(T + col * pc.nv + v), s);
    }
    float *dst = c + (ip * pc.st_p + iq * pc.st_q + (long long)lb * pc.st_b);
    *dst = ADD ? *dst + s : s;
}

// ---------------------------------------------------------------- host side
namespace {
std::mutex g_plane_mu;

// centred cardinal B-spline of degree n (FP64), half-open box for n = 0
double bspline(int n, double x)
{
    const double a = fabs(x);
    switch (n) {
    case 0: return (x >= -0.5 && x < 0.5) ? 1.0 : 0.0;
    case 1: return a < 1.0 ? 1.0 - a : 0.0;
    case 2: return a < 0.5 ? 0.75 - a * a : (a < 1.5 ? 0.5 * (1.5 - a) * (1.5 - a) : 0.0);
    default:
        if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
        if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    }
}

PlaneCall call_of(const spl_geometry *g)
{
    const PlaneGroup &pg = *g->plane;
    const DevGeom &dg = g->dev;
    const long long st[3] = {1, dg.n[0], (long long)dg.n[0] * dg.n[1]};
    PlaneCall pc;
    pc.n_p = dg.n[pg.p];
    pc.n_q = dg.n[pg.q];
    pc.n_b = dg.n[pg.b];
    pc.st_p = st[pg.p];
    pc.st_q = st[pg.q];
    pc.st_b = st[pg.b];
    pc.ncol = pg.ncol;
    pc.rows = pg.rows;
    pc.nu = dg.nu;
    pc.nv = dg.nv;
    return pc;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int N>
spl_status build_pack(spl_geometry *g, cudaStream_t st)
{
    PlaneGroup &pg = *g->plane;
    PlanePack &pk = pg.pack[N];
    const DevGeom &dg = g->dev;
    const int nv = dg.nv, nb = dg.n[pg.b];
    constexpr double W = 0.5 * (N + 1);
    // b weights of the detector rows (FP64 on the host)
    std::vector<int> lb0(nv), vr(2 * (size_t)nb);
    std::vector<float> wz((size_t)nv * (N + 1));
    for (int l = 0; l < nb; ++l) {
        vr[2 * l] = nv;
        vr[2 * l + 1] = -1;
    }
    for (int v = 0; v < nv; ++v) {
        const double z = pg.z0 + v * pg.dz;
        const double fl = floor(z + W);
        lb0[v] = (int)fmax(fmin(fl - N, 1e9), -1e9);
        for (int i = 0; i <= N; ++i) {
            const long long l = (long long)lb0[v] + i;
            wz[(size_t)v * (N + 1) + i] = (float)bspline(N, z - (double)l);
            if (l >= 0 && l < nb) {
                if (v < vr[2 * l]) vr[2 * l] = v;
                if (v > vr[2 * l + 1]) vr[2 * l + 1] = v;
            }
        }
    }
    // first allocation: everything but the nnz-sized arrays
    const size_t o_rp = 0;
    const size_t o_cp = align256(o_rp + (pg.rows + 1) * sizeof(long long));
    const size_t o_lb = align256(o_cp + (pg.ncol + 1) * sizeof(long long));
    const size_t o_wz = align256(o_lb + nv * sizeof(int));
    const size_t o_vr = align256(o_wz + wz.size() * sizeof(float));
    const size_t o_S = align256(o_vr + vr.size() * sizeof(int));
    const size_t o_T = align256(o_S + pg.ncol * nv * sizeof(float));
    const size_t o_yt = align256(o_T + pg.ncol * nv * sizeof(float));
    const size_t o_cur = align256(o_yt + pg.rows * nv * sizeof(float));
    const size_t bytes1 = align256(o_cur + (pg.ncol + 1) * sizeof(long long));
    char *b1 = nullptr;
    if (cudaMalloc(&b1, bytes1) != cudaSuccess) {
        cudaGetLastError();
        pk.state = -1;
        return fail(SPL_ERR_OOM, "plane matrices: cudaMalloc(%zu) failed", bytes1);
    }
    pk.block = b1;
    pk.row_ptr = (long long *)(b1 + o_rp);
    pk.col_ptr = (long long *)(b1 + o_cp);
    pk.lb0 = (int *)(b1 + o_lb);
    pk.wz = (float *)(b1 + o_wz);
    pk.vr = (int *)(b1 + o_vr);
    pk.S = (float *)(b1 + o_S);
    pk.T = (float *)(b1 + o_T);
    pk.yt = (float *)(b1 + o_yt);
    long long *cursor = (long long *)(b1 + o_cur);
    spl_status s = cuda_check(cudaMemcpyAsync(pk.lb0, lb0.data(), nv * sizeof(int), cudaMemcpyHostToDevice, st), "plane upload");
    if (s == SPL_OK)
        s = cuda_check(cudaMemcpyAsync(pk.wz, wz.data(), wz.size() * sizeof(float), cudaMemcpyHostToDevice, st),
                       "plane upload");
    if (s == SPL_OK)
        s = cuda_check(cudaMemcpyAsync(pk.vr, vr.data(), vr.size() * sizeof(int), cudaMemcpyHostToDevice, st),
                       "plane upload");
    PlaneArgs pa;
    pa.n_p = dg.n[pg.p];
    pa.b = pg.b;
    pa.nu = dg.nu;
    pa.rows = pg.rows;
    const QuadRule qr = quad_rule(N);
    const unsigned rb = (unsigned)((pg.rows + 127) / 128);
    if (s == SPL_OK) {
        k_plane_rows<N, false><<<rb, 128, 0, st>>>(dg, pa, pk.row_ptr, nullptr, nullptr, qr);
        k_scan<<<1, 1024, 0, st>>>(pk.row_ptr, pg.rows);
        s = cuda_check(cudaGetLastError(), "plane row count");
    }
    long long nnz = 0;
    if (s == SPL_OK)
        s = cuda_check(cudaMemcpyAsync(&nnz, pk.row_ptr + pg.rows, sizeof(long long), cudaMemcpyDeviceToHost, st),
                       "plane nnz");
    if (s == SPL_OK) s = cuda_check(cudaStreamSynchronize(st), "plane nnz");
    char *b2 = nullptr;
    const size_t bytes2 = align256((size_t)nnz * (2 * sizeof(int) + 2 * sizeof(float))) + 256;
    if (s == SPL_OK && cudaMalloc(&b2, bytes2) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b1);
        pk.block = nullptr;
        pk.state = -1;
        return fail(SPL_ERR_OOM, "plane matrices: cudaMalloc(%zu) failed", bytes2);
    }
    if (s != SPL_OK) {
        cudaFree(b1);
        pk.block = nullptr;
        pk.state = -1;
        return s;
    }
    pk.block2 = b2;
    pk.nnz = nnz;
    pk.row_col = (int *)b2;
    pk.row_val = (float *)(b2 + align256((size_t)nnz * sizeof(int)));
    pk.col_row = (int *)((char *)pk.row_val + align256((size_t)nnz * sizeof(float)));
    pk.col_val = (float *)((char *)pk.col_row + align256((size_t)nnz * sizeof(int)));
    k_plane_rows<N, true><<<rb, 128, 0, st>>>(dg, pa, pk.row_ptr, pk.row_col, pk.row_val, qr);
    s = cuda_check(cudaMemsetAsync(pk.col_ptr, 0, (pg.ncol + 1) * sizeof(long long), st), "plane columns");
    if (s == SPL_OK) {
        k_plane_colcount<<<rb, 128, 0, st>>>(pg.rows, pk.row_ptr, pk.row_col, pk.col_ptr);
        k_scan<<<1, 1024, 0, st>>>(pk.col_ptr, pg.ncol);
        s = cuda_check(cudaGetLastError(), "plane columns");
    }
    if (s == SPL_OK)
        s = cuda_check(cudaMemcpyAsync(cursor, pk.col_ptr, (pg.ncol + 1) * sizeof(long long), cudaMemcpyDeviceToDevice, st),
                       "plane columns");
    if (s == SPL_OK) {
        k_plane_colfill<<<rb, 128, 0, st>>>(pg.rows, pk.row_ptr, pk.row_col, pk.row_val, cursor, pk.col_row, pk.col_val);
        s = cuda_check(cudaGetLastError(), "plane columns");
    }
    if (s == SPL_OK) s = cuda_check(cudaStreamSynchronize(st), "plane build");
    if (s != SPL_OK) {
        cudaFree(b2);
        cudaFree(b1);
        pk.block = pk.block2 = nullptr;
        pk.state = -1;
        return s;
    }
    pk.state = 1;
    return SPL_OK;
}
}  // namespace

bool plane_ready(spl_geometry *g, int degree, cudaStream_t st, spl_status *err)
{
    *err = SPL_OK;
    if (!g->plane || degree < 0 || degree > 3) return false;
    std::lock_guard<std::mutex> lock(g_plane_mu);
    PlanePack &pk = g->plane->pack[degree];
    if (pk.state == 0) {
        switch (degree) {
        case 0: *err = build_pack<0>(g, st); break;
        case 1: *err = build_pack<1>(g, st); break;
        case 2: *err = build_pack<2>(g, st); break;
        default: *err = build_pack<3>(g, st); break;
        }
    }
    return pk.state == 1;
}

int plane_state(const spl_geometry *g, int degree)
{
    if (!g->plane || degree < 0 || degree > 3) return -1;
    std::lock_guard<std::mutex> lock(g_plane_mu);
    return g->plane->pack[degree].state;
}

void plane_free(PlaneGroup *pg)
{
    if (!pg) return;
    for (int n = 0; n < 4; ++n) {
        if (pg->pack[n].block2) cudaFree(pg->pack[n].block2);
        if (pg->pack[n].block) cudaFree(pg->pack[n].block);
    }
    if (pg->join) cudaEventDestroy(pg->join);
    if (pg->fork) cudaEventDestroy(pg->fork);
    if (pg->side) cudaStreamDestroy(pg->side);
    delete pg;
}

template <int N>
static spl_status plane_forward_n(const spl_geometry *g, int kahan, const float *c, float *y, cudaStream_t st)
{
    const PlaneGroup &pg = *g->plane;
    const PlanePack &pk = pg.pack[N];
    const PlaneCall pc = call_of(g);
    const long long nz = pc.ncol * pc.nv;
    k_plane_zres<N><<<(unsigned)((nz + 255) / 256), 256, 0, st>>>(pc, c, pk.lb0, pk.wz, pk.S);
    const unsigned blocks = (unsigned)((pg.rows + kPlaneWarps - 1) / kPlaneWarps);
    if (kahan)
        k_plane_gather<true, true><<<blocks, 32 * kPlaneWarps, 0, st>>>(pg.rows, pk.row_ptr, pk.row_col, pk.row_val, pk.S,
                                                                        y, pc.nv, pc.nu, g->dev.view_order);
    else
        k_plane_gather<false, true><<<blocks, 32 * kPlaneWarps, 0, st>>>(pg.rows, pk.row_ptr, pk.row_col, pk.row_val,
                                                                         pk.S, y, pc.nv, pc.nu, g->dev.view_order);
    return cuda_check(cudaGetLastError(), "plane forward launch");
}

// the adjoint's first stage: y transposed per view, then T = column gather
template <int N>
static spl_status plane_adjoint_t_n(const spl_geometry *g, const float *y, cudaStream_t st)
{
    const PlaneGroup &pg = *g->plane;
    const PlanePack &pk = pg.pack[N];
    const PlaneCall pc = call_of(g);
    dim3 tg((pc.nu + 31) / 32, (pc.nv + 31) / 32, pg.n_views);
    k_plane_ytrans<<<tg, 256, 0, st>>>(y, pk.yt, g->dev.view_order, pc.nu, pc.nv);
    const unsigned blocks = (unsigned)((pg.ncol + kPlaneWarps - 1) / kPlaneWarps);
    k_plane_gather<true, false><<<blocks, 32 * kPlaneWarps, 0, st>>>(pg.ncol, pk.col_ptr, pk.col_row, pk.col_val, pk.yt,
                                                                     pk.T, pc.nv, pc.nu, nullptr);
    return cuda_check(cudaGetLastError(), "plane adjoint launch");
}

// the adjoint's second stage: c from T (written, or added with ADD)
template <int N, bool ADD>
static spl_status plane_adjoint_c_n(const spl_geometry *g, float *c, cudaStream_t st)
{
    const PlanePack &pk = g->plane->pack[N];
    const PlaneCall pc = call_of(g);
    const long long nc = pc.ncol * pc.n_b;
    k_plane_zadj<N, ADD><<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(pc, pk.T, pk.lb0, pk.wz, pk.vr, c);
    return cuda_check(cudaGetLastError(), "plane adjoint launch");
}

template <int N>
static spl_status plane_adjoint_n(const spl_geometry *g, const float *y, float *c, cudaStream_t st)
{
    spl_status s = plane_adjoint_t_n<N>(g, y, st);
    if (s != SPL_OK) return s;
    return plane_adjoint_c_n<N, false>(g, c, st);
}

spl_status plane_forward(const spl_geometry *g, int degree, int kahan, const float *c, float *y, cudaStream_t st)
{
    switch (degree) {
    case 0: return plane_forward_n<0>(g, kahan, c, y, st);
    case 1: return plane_forward_n<1>(g, kahan, c, y, st);
    case 2: return plane_forward_n<2>(g, kahan, c, y, st);
    default: return plane_forward_n<3>(g, kahan, c, y, st);
    }
}

spl_status plane_adjoint(const spl_geometry *g, int degree, const float *y, float *c, cudaStream_t st)
{
    switch (degree) {
    case 0: return plane_adjoint_n<0>(g, y, c, st);
    case 1: return plane_adjoint_n<1>(g, y, c, st);
    case 2: return plane_adjoint_n<2>(g, y, c, st);
    default: return plane_adjoint_n<3>(g, y, c, st);
    }
}

spl_status plane_adjoint_t(const spl_geometry *g, int degree, const float *y, cudaStream_t st)
{
    switch (degree) {
    case 0: return plane_adjoint_t_n<0>(g, y, st);
    case 1: return plane_adjoint_t_n<1>(g, y, st);
    case 2: return plane_adjoint_t_n<2>(g, y, st);
    default: return plane_adjoint_t_n<3>(g, y, st);
    }
}

spl_status plane_adjoint_add(const spl_geometry *g, int degree, float *c, cudaStream_t st)
{
    switch (degree) {
    case 0: return plane_adjoint_c_n<0, true>(g, c, st);
    case 1: return plane_adjoint_c_n<1, true>(g, c, st);
    case 2: return plane_adjoint_c_n<2, true>(g, c, st);
    default: return plane_adjoint_c_n<3, true>(g, c, st);
    }
}

}  // namespace spl

extern "C" spl_status spl_prepare(spl_geometry *g, const spl_basis_desc *basis, void *stream)
{
    spl::clear_error();
    if (!g) return spl::fail(SPL_ERR_ARG, "geometry is NULL");
    spl_status s = spl::check_basis(basis);
    if (s != SPL_OK) return s;
    if (basis->mode == SPL_FP_MLP) return SPL_OK;
    if (basis->mode == SPL_FP_TABLE) return spl::table_build(g, basis->degree, (cudaStream_t)stream);
    if (basis->separable == SPL_SEP_OFF) return SPL_OK;
    spl_status err;
    spl::plane_ready(g, basis->degree, (cudaStream_t)stream, &err);
    return err;
}
