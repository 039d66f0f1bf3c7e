// project.cu -- forward projection A (Algorithm 2, Eq. 4) and its matched
// adjoint A^T (Sec. 2.3: the adjoint is matched exactly to the forward),
// exact quadrature footprint.
//
// Forward: one thread per ray; the 128 threads of a block cover a 16 x 8
// detector tile of one view (a warp is an 8 x 4 sub-tile), so neighbouring
// lanes walk neighbouring lines and gather neighbouring coefficients (L1
// hits).  Each ray is walked with the cell march (one Gauss node set per
// point of the ray, an (n+1)^3 register window); the per-cell partial sums
// are added along the ray with Kahan compensation.
//
// Adjoint, view geometries, two forms that visit the same pairs with the
// same footprint values:
//  * scatter (default): the forward's thread mapping; each flushed
//    contribution y_r * P is added to c with a float atomic (a
//    fire-and-forget reduction in L2), which overlaps with the FP32 work --
//    on GB300 A^T then costs about as much as A;
//  * gather: one block per 16^3 coefficient brick; for every batch of 8
//    views the block projects the brick's support box onto the detectors,
//    walks the rays of those pixel windows through the brick's cells with
//    the same set-up and cell march, accumulates y_r * P in shared memory
//    and folds the batch into FP64 totals; no global atomics, each
//    coefficient written once.
// Adjoint, explicit rays: no view structure to gather over: scatter.
#include <stdio.h>
#include <string.h>

#include "spl_host.h"
#include "spl_mlp.cuh"

namespace spl {

// ---------------------------------------------------------------- sinks
// Sinks take a basis either by index (flush, the flat cell march) or by its
// offset in the sink's layout, off + l_d S0 + l_a S1 + l_b S2 in unsigned
// (wrapping) arithmetic, with a flag that it lies in the region (put, the
// piece march).
struct FwdSink {
    static constexpr bool plane = false;
    static constexpr bool face = false;
    const float *__restrict__ c;
    int S0, S1, S2;
    unsigned off;
    SinkBox bx;
    float inv_wd;
    bool kahan;
    // the cell's partial sum c_l * F_l, spread over four independent
    // accumulators (a face's 16 gathers and FMAs then form four chains of
    // four instead of one chain of sixteen)
    float acc[4], sum, comp;
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return bx.meets(d0, d1, a0, a1, b0, b1);
    }
    __device__ __forceinline__ void flush(int ld, int la, int lb, float v)
    {
        if (bx.holds(ld, la, lb)) acc[0] = fmaf(__ldg(c + (ld * S0 + la * S1 + lb * S2)), v, acc[0]);
    }
    __device__ __forceinline__ float wscale() const { return 1.0f; }
    __device__ __forceinline__ void put(unsigned o, bool in, float v, int slot)
    {
        if (in) acc[slot & 3] = fmaf(__ldg(c + o), v, acc[slot & 3]);
    }
    __device__ __forceinline__ void cell_end()
    {
        const float v = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * inv_wd;
        acc[0] = acc[1] = acc[2] = acc[3] = 0.0f;
        if (kahan) kahan_add(sum, comp, v);
        else sum += v;
    }
};

struct CountSink {
    static constexpr bool plane = false;
    static constexpr bool face = false;
    int S0, S1, S2;
    unsigned off;
    SinkBox bx;
    unsigned int n;       // bases with a nonzero footprint
    unsigned int pieces;  // integrated pieces (GL nodes each)
    __device__ __forceinline__ void piece() { ++pieces; }
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return bx.meets(d0, d1, a0, a1, b0, b1);
    }
    __device__ __forceinline__ void flush(int ld, int la, int lb, float v)
    {
        n += (bx.holds(ld, la, lb) && v > 0.0f) ? 1u : 0u;
    }
    __device__ __forceinline__ float wscale() const { return 1.0f; }
    __device__ __forceinline__ void put(unsigned, bool in, float v, int) { n += (in && v > 0.0f) ? 1u : 0u; }
    __device__ __forceinline__ void cell_end() {}
};

// adjoint, scatter: y_r / |w_d| * F_l added to c_l with a float atomic.
// The target of a piece-marched ray is a set of four shifted copies of a
// layout of c (copy j holds coefficient i at position j * cs + i + j, cs a
// multiple of 4): a face row of N+1 = 4 consecutive floats starting at
// index lo goes, as one 16-byte vector atomic, to the copy j = -lo mod 4 in
// which it starts a 16-byte group.  Faces without such a row, the cell
// march's flushes and the last window take scalar atomics into copy 0.
// The copies are summed into c afterwards (k_fold_copies*).
struct AtomicSink {
    static constexpr bool plane = false;
    static constexpr bool face = true;
    float *__restrict__ c;  // copy 0 (or c itself where no vector row is written)
    size_t cs;              // copy stride in floats
    int S0, S1, S2;
    unsigned off;
    SinkBox bx;
    float yv;
    // w0..w3 (already scaled) at p, p + s, p + 2 s, p + 3 s with s = +1 (UP)
    // or -1: one aligned 16-byte atomic into the copy where the run starts
    // a group
    template <bool UP>
    __device__ __forceinline__ void row4(unsigned p, float w0, float w1, float w2, float w3)
    {
        const unsigned lo = UP ? p : p - 3u;
        const unsigned j = (0u - lo) & 3u;
        const float4 f = UP ? make_float4(w0, w1, w2, w3) : make_float4(w3, w2, w1, w0);
        atomicAdd(reinterpret_cast<float4 *>(c + ((size_t)j * cs + (size_t)(lo + j))), f);
    }
    // the face's (N+1)^2 values at base + x SX + y SY.  In the layout of a
    // piece-marched ray the b axis is contiguous (S2 = +-1), so the faces of
    // d and a events (SY = S2) have rows along y; the faces of b events
    // (SY = S1) take scalar atomics.  The sign of S2 is the ray's and
    // mostly the warp's, so the two row directions are branches.
    template <int N>
    __device__ __forceinline__ void put_face(unsigned base, unsigned SX, unsigned SY, const float (&v)[N + 1][N + 1])
    {
        if constexpr (N == 3) {
            if (SY == 1u) {
#pragma unroll
                for (int x = 0; x <= N; ++x) row4<true>(base + (unsigned)x * SX, v[x][0], v[x][1], v[x][2], v[x][3]);
                return;
            }
            if (SY == 0xffffffffu) {
#pragma unroll
                for (int x = 0; x <= N; ++x) row4<false>(base + (unsigned)x * SX, v[x][0], v[x][1], v[x][2], v[x][3]);
                return;
            }
        }
#pragma unroll
        for (int x = 0; x <= N; ++x)
#pragma unroll
            for (int y = 0; y <= N; ++y) atomicAdd(c + (base + (unsigned)x * SX + (unsigned)y * SY), v[x][y]);
    }
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return bx.meets(d0, d1, a0, a1, b0, b1);
    }
    __device__ __forceinline__ void flush(int ld, int la, int lb, float v)
    {
        if (bx.holds(ld, la, lb)) atomicAdd(c + (ld * S0 + la * S1 + lb * S2), yv * v);
    }
    // the piece march scales its Gauss weights by y_r (wscale), so the
    // window values that reach put and put_face already carry the factor
    __device__ __forceinline__ float wscale() const { return yv; }
    __device__ __forceinline__ void put(unsigned o, bool in, float v, int)
    {
        if (in) atomicAdd(c + o, v);
    }
    __device__ __forceinline__ void cell_end() {}
};

// brick of the gather adjoint: the region is the brick, the target the
// shared-memory brick array (mirrored strides S0..S2, offset off)
struct BrickSink {
    static constexpr bool plane = false;
    static constexpr bool face = false;
    float *part;
    int S0, S1, S2;
    unsigned off;
    SinkBox bx;
    float yv;
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return bx.meets(d0, d1, a0, a1, b0, b1);
    }
    __device__ __forceinline__ void flush(int ld, int la, int lb, float v)
    {
        if (bx.holds(ld, la, lb)) atomicAdd(part + (unsigned)(ld * S0 + la * S1 + lb * S2 + (int)off), yv * v);
    }
    __device__ __forceinline__ float wscale() const { return 1.0f; }
    __device__ __forceinline__ void put(unsigned o, bool in, float v, int)
    {
        if (in) atomicAdd(part + o, yv * v);
    }
    __device__ __forceinline__ void cell_end() {}
};

// ---------------------------------------------------------------- forward

// View classes of a view-kernel launch.  VM_FLAT / VM_GENERAL: parallel
// views of one class, taken from the geometry's view order; the form is
// fixed at compile time, so each kernel carries the registers of one form
// only (a parallel view's rays share their direction, hence their form).
// VM_CONE: cone views, every ray with the piece march (a cone ray with a
// zero direction component, rare, is integrated by the general form too:
// its constant factor is then evaluated at every node, which is exact but
// slower; the kernel keeps the registers and code of one form).  VM_RAYS:
// explicit rays, the form chosen per ray.
enum { VM_CONE = 0, VM_FLAT = 1, VM_GENERAL = 2, VM_RAYS = 3 };

template <int N, int VM, class Sink>
__device__ __forceinline__ bool march_vm(const RaySetup &rs, int cf, int cl, const QuadRule &qr, Sink &sk)
{
    if constexpr (VM == VM_FLAT) return cell_march<N, Sink, true>(rs, cf, cl, qr, sk);
    else if constexpr (VM == VM_GENERAL || VM == VM_CONE) return piece_march<N, Sink>(rs, cf, cl, qr, sk);
    else return march<N>(rs, cf, cl, qr, sk);
}

// The march form of a ray of geometry kind `kind` (used where one kernel
// serves every view kind: the pair count and the brick adjoint), the same
// as the projection kernels': cone rays always take the piece march.
template <int N, class Sink>
__device__ __forceinline__ bool march_kind(int kind, const RaySetup &rs, int cf, int cl, const QuadRule &qr, Sink &sk)
{
    if (kind == SPL_CONE) return piece_march<N, Sink>(rs, cf, cl, qr, sk);
    return march<N>(rs, cf, cl, qr, sk);
}

// blocks per SM the register budget is sized for (measured): the flat form
// needs an (n+1)^2 window, the general one (n+1)^3 accumulators plus the
// flush state (3 blocks x 168 registers; 4 x 128 spills and is slower); the
// direct march keeps (n+1)^3 coefficients but no flush state (4 x 128)
template <int VM, bool DIRECT = false> struct ViewBlocks {
    static constexpr int value = VM == VM_FLAT ? 6 : (DIRECT ? 4 : 3);
};

// DIRECT: rays with three nonzero direction components take the direct
// march (the line integral of f itself); flat rays keep the footprint form
template <int N, int VM, bool DIRECT = false>
__device__ __forceinline__ float march_forward(const RaySetup &rs, const float *__restrict__ c, const QuadRule &qr,
                                               bool kahan, int *err)
{
    if constexpr (DIRECT && VM != VM_FLAT) {
        if (VM == VM_GENERAL || VM == VM_CONE || rs.rb != 0.0f) {
            float out;
            if (!direct_march<N>(rs, c, rs.S[0], rs.S[1], rs.S[2], make_box(rs.lo, rs.hi), qr, kahan, out))
                atomicOr(err, 1);
            return out;
        }
    }
    FwdSink sk;
    sk.c = c;
    sk.S0 = rs.S[0];
    sk.S1 = rs.S[1];
    sk.S2 = rs.S[2];
    sk.off = 0u;
    sk.bx = make_box(rs.lo, rs.hi);
    sk.inv_wd = rs.inv_wd;
    sk.kahan = kahan;
    sk.acc[0] = sk.acc[1] = sk.acc[2] = sk.acc[3] = sk.sum = sk.comp = 0.0f;
    if (!march_vm<N, VM>(rs, rs.c0, rs.c1, qr, sk)) atomicOr(err, 1);
    return sk.sum;
}

// cone views (every ray with the piece march)
template <int N, bool DIRECT>
__global__ void __launch_bounds__(128, (ViewBlocks<VM_CONE, DIRECT>::value))
    k_forward_views(DevGeom g, const float *__restrict__ c, float *__restrict__ y, QuadRule qr, int kahan)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const int k = blockIdx.z;
    if (iu >= g.nu || iv >= g.nv) return;
    RaySetup rs;
    float v = 0.0f;
    if (view_setup<N>(g, grid_of(g), k, iu, iv, rs))
        v = march_forward<N, VM_CONE, DIRECT>(rs, c, qr, kahan != 0, g.err);
    y[((long long)k * g.nv + iv) * g.nu + iu] = v;
}

// parallel views of one class (VM_FLAT or VM_GENERAL): view blockIdx.z of
// the chunk
template <int N, int VM, bool DIRECT>
__global__ void __launch_bounds__(128, (ViewBlocks<VM, DIRECT>::value))
    k_forward_pviews(DevGeom g, const float *__restrict__ c, float *__restrict__ y, QuadRule qr, int kahan,
                     const __grid_constant__ ViewChunk vc)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const ViewConst &V = vc.v[blockIdx.z];
    const int k = V.view;
    if (iu >= g.nu || iv >= g.nv) return;
    RaySetup rs;
    float v = 0.0f;
    if (view_setup<N>(g, grid_of(g), k, iu, iv, rs)) {
        use_view_const(V, rs);
        v = march_forward<N, VM, DIRECT>(rs, c, qr, kahan != 0, g.err);
    }
    y[((long long)k * g.nv + iv) * g.nu + iu] = v;
}

template <int N, bool DIRECT>
__global__ void __launch_bounds__(128) k_forward_rays(DevGeom g, const float *__restrict__ c, float *__restrict__ y,
                                                      QuadRule qr, int kahan)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.n_rays) return;
    double s[3], w[3];
    explicit_ray(g, r, s, w);
    RaySetup rs;
    float v = 0.0f;
    if (ray_setup<N>(grid_of(g), s, w, rs)) v = march_forward<N, VM_RAYS, DIRECT>(rs, c, qr, kahan != 0, g.err);
    y[r] = v;
}

// ---------------------------------------------------------------- pair count
template <int N>
__device__ __forceinline__ void march_count(int kind, const RaySetup &rs, const QuadRule &qr, int *err,
                                            unsigned int &pairs, unsigned int &pieces, unsigned int &flat_pieces)
{
    CountSink sk;
    sk.S0 = sk.S1 = sk.S2 = 0;
    sk.off = 0u;
    sk.bx = make_box(rs.lo, rs.hi);
    sk.n = 0u;
    sk.pieces = 0u;
    if (!march_kind<N>(kind, rs, rs.c0, rs.c1, qr, sk)) atomicOr(err, 1);
    const bool flat = rs.rb == 0.0f && kind != SPL_CONE;
    pairs = sk.n;  // (nonzero FP32 footprints; the contributions come from the exact count)
    pieces = flat ? 0u : sk.pieces;
    flat_pieces = flat ? sk.pieces : 0u;
}

__device__ __forceinline__ void add_count(unsigned long long *count, unsigned int v)
{
    unsigned long long x = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(count, x);
}

template <int N>
__global__ void __launch_bounds__(128) k_count_views(DevGeom g, unsigned long long *count, QuadRule qr)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const int k = blockIdx.z;
    unsigned int v = 0, pc = 0, pf = 0;
    RaySetup rs;
    if (iu < g.nu && iv < g.nv && view_setup<N>(g, grid_of(g), k, iu, iv, rs))
        march_count<N>(g.kind, rs, qr, g.err, v, pc, pf);
    add_count(count + 1, pc);
    add_count(count + 2, pf);
}

template <int N>
__global__ void __launch_bounds__(128) k_count_rays(DevGeom g, unsigned long long *count, QuadRule qr)
{
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int v = 0, pc = 0, pf = 0;
    if (r < g.n_rays) {
        double s[3], w[3];
        explicit_ray(g, r, s, w);
        RaySetup rs;
        if (ray_setup<N>(grid_of(g), s, w, rs)) march_count<N>(SPL_RAYS, rs, qr, g.err, v, pc, pf);
    }
    add_count(count + 1, pc);
    add_count(count + 2, pf);
}

// ---------------------------------------------------------------- adjoint: ray-driven scatter

template <int N, int VM>
__device__ __forceinline__ void scatter_ray(const RaySetup &rs, float yr, float *__restrict__ c, size_t cs,
                                            const QuadRule &qr, int *err)
{
    AtomicSink sk;
    sk.c = c;
    sk.cs = cs;
    sk.S0 = rs.S[0];
    sk.S1 = rs.S[1];
    sk.S2 = rs.S[2];
    sk.off = 0u;
    sk.bx = make_box(rs.lo, rs.hi);
    sk.yv = yr * rs.inv_wd;
    if (!march_vm<N, VM>(rs, rs.c0, rs.c1, qr, sk)) atomicOr(err, 1);
}

// The layout a piece-marched scatter ray reduces into: the one whose
// contiguous axis is the ray's b axis (its smallest direction component),
// l0 = [z][y][x] (x fast), l1 = [z][x][y] (y fast) or l2 = [y][x][z] (z
// fast), each as four shifted copies (AtomicSink); rs.S is re-pointed at
// that layout.  The faces that leave the window on d and a events (all but
// the rare b events) then contain rows along b and go out as one 16-byte
// vector atomic per row, and the lanes of a warp, whose rays lie side by
// side, reduce into neighbouring addresses.  The copies are folded into c
// after the launch.
__device__ __forceinline__ float *b_fast_target(const DevGeom &g, RaySetup &rs, float *l0, float *l1, float *l2)
{
    if (rs.ax[2] == 0) return l0;
    int st[3];
    float *t;
    if (rs.ax[2] == 1) {
        st[0] = g.n[1];
        st[1] = 1;
        st[2] = g.n[0] * g.n[1];
        t = l1;
    } else {
        st[0] = g.n[2];
        st[1] = g.n[0] * g.n[2];
        st[2] = 1;
        t = l2;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) rs.S[q] = rs.sg[q] * st[rs.ax[q]];
    return t;
}

// rays r0 .. r1-1
template <int N>
__global__ void __launch_bounds__(128) k_adjoint_rays(DevGeom g, const float *__restrict__ y, float *__restrict__ l0,
                                                      float *__restrict__ l1, float *__restrict__ l2, QuadRule qr,
                                                      long long r0, long long r1)
{
    const long long r = r0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= r1) return;
    const float yr = y[r];
    if (yr == 0.0f) return;
    double s[3], w[3];
    explicit_ray(g, r, s, w);
    RaySetup rs;
    if (!ray_setup<N>(grid_of(g), s, w, rs)) return;
    float *t = b_fast_target(g, rs, l0, l1, l2);
    scatter_ray<N, VM_RAYS>(rs, yr, t, g.lay_cs, qr, g.err);
}

// view geometries, scatter form: the forward's thread mapping; views
// v0 + blockIdx.z
template <int N>
__global__ void __launch_bounds__(128, 3)
    k_adjoint_views_scatter(DevGeom g, const float *__restrict__ y, float *__restrict__ l0, float *__restrict__ l1,
                            float *__restrict__ l2, QuadRule qr, int v0)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const int k = v0 + blockIdx.z;
    if (iu >= g.nu || iv >= g.nv) return;
    const float yr = __ldg(y + ((long long)k * g.nv + iv) * g.nu + iu);
    if (yr == 0.0f) return;
    RaySetup rs;
    if (!view_setup<N>(g, grid_of(g), k, iu, iv, rs)) return;
    float *t = b_fast_target(g, rs, l0, l1, l2);
    scatter_ray<N, VM_CONE>(rs, yr, t, g.lay_cs, qr, g.err);
}

// c[i] += sum_j l0[j cs + i + j]: the fold of the x-fast copies into c
__global__ void k_fold_copies(float *__restrict__ c, const float *__restrict__ in, long long n, long long cs)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        c[i] += (in[i] + in[cs + i + 1]) + (in[2 * cs + i + 2] + in[3 * cs + i + 3]);
}

// out[s][r][q] += sum_j in[j cs + (s Q + q) R + r + j]: the fold of the
// shifted copies of a Q x R row-major layout into c, slab by slab.  y fast:
// slabs z, Q = nx, R = ny; z fast: one slab, Q = nx ny, R = nz.  32 x 32
// tiles through shared memory, both sides coalesced.
__global__ void __launch_bounds__(256) k_fold_copies_transpose(float *__restrict__ out, const float *__restrict__ in,
                                                               long long Q, long long R, long long slabs, long long cs)
{
    __shared__ float t[32][33];
    const long long q0 = (long long)blockIdx.x * 32, r0 = (long long)blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (long long sl = blockIdx.z; sl < slabs; sl += gridDim.z) {
        const long long base = sl * Q * R;
        for (int j = ty; j < 32; j += 8) {
            const long long q = q0 + j, r = r0 + tx;
            float v = 0.0f;
            if (q < Q && r < R) {
                const long long i = base + q * R + r;
                v = (in[i] + in[cs + i + 1]) + (in[2 * cs + i + 2] + in[3 * cs + i + 3]);
            }
            t[j][tx] = v;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const long long r = r0 + j, q = q0 + tx;
            if (q < Q && r < R) out[base + r * Q + q] += t[tx][j];
        }
        __syncthreads();
    }
}

// parallel views of one class; the general class (piece march) reduces
// into the view's b-fast layout (ViewConst::lay, Sb), the flat class (cell
// march, scalar atomics) into c
template <int N, int VM>
__global__ void __launch_bounds__(128, ViewBlocks<VM>::value)
    k_adjoint_pviews_scatter(DevGeom g, const float *__restrict__ y, float *__restrict__ c, float *__restrict__ l0,
                             float *__restrict__ l1, float *__restrict__ l2, QuadRule qr,
                             const __grid_constant__ ViewChunk vc)
{
    int iu, iv;
    tile_pixel(iu, iv);
    const ViewConst &V = vc.v[blockIdx.z];
    const int k = V.view;
    if (iu >= g.nu || iv >= g.nv) return;
    const float yr = __ldg(y + ((long long)k * g.nv + iv) * g.nu + iu);
    if (yr == 0.0f) return;
    RaySetup rs;
    if (view_setup<N>(g, grid_of(g), k, iu, iv, rs)) {
        use_view_const(V, rs);
        if constexpr (VM == VM_GENERAL) {
            float *t = V.lay == 0 ? l0 : (V.lay == 1 ? l1 : l2);
#pragma unroll
            for (int q = 0; q < 3; ++q) rs.S[q] = V.Sb[q];
            scatter_ray<N, VM>(rs, yr, t, g.lay_cs, qr, g.err);
        } else {
            scatter_ray<N, VM>(rs, yr, c, 0, qr, g.err);
        }
    }
}

// ---------------------------------------------------------------- adjoint: brick gather (view geometries)
constexpr int kBrick = 16;                        // brick edge (coefficients)
constexpr int kBrickVol = kBrick * kBrick * kBrick;
constexpr int kAdjThreads = 256;
constexpr int kViewBatch = 8;                     // views per shared-memory fold

// detector pixel window of the box [lo, hi] (world) for view k: projection
// of its 8 corners (parallel: along the direction; cone: from the source)
__device__ __forceinline__ bool pixel_window(const DevGeom &g, int k, const double (&lo)[3], const double (&hi)[3],
                                             int &u0, int &u1, int &v0, int &v1)
{
    const ViewPose &P = g.views[k];
    double amin = 1e300, amax = -1e300, bmin = 1e300, bmax = -1e300;
    const double cu = 0.5 * (g.nu - 1), cv = 0.5 * (g.nv - 1);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        double x[3] = {(corner & 1) ? hi[0] : lo[0], (corner & 2) ? hi[1] : lo[1], (corner & 4) ? hi[2] : lo[2]};
        double pt[3];
        if (g.kind == 1) {
            // move x along the direction onto the detector plane
            double rel[3] = {x[0] - P.dc[0], x[1] - P.dc[1], x[2] - P.dc[2]};
            const double t = (rel[0] * P.nrm[0] + rel[1] * P.nrm[1] + rel[2] * P.nrm[2]) /
                             (P.src[0] * P.nrm[0] + P.src[1] * P.nrm[1] + P.src[2] * P.nrm[2]);
#pragma unroll
            for (int e = 0; e < 3; ++e) pt[e] = rel[e] - t * P.src[e];
        } else {
            double dx[3] = {x[0] - P.src[0], x[1] - P.src[1], x[2] - P.src[2]};
            double sd[3] = {P.dc[0] - P.src[0], P.dc[1] - P.src[1], P.dc[2] - P.src[2]};
            const double num = sd[0] * P.nrm[0] + sd[1] * P.nrm[1] + sd[2] * P.nrm[2];
            const double den = dx[0] * P.nrm[0] + dx[1] * P.nrm[1] + dx[2] * P.nrm[2];
            if (!(den * num > 0.0)) return true;  // corner behind the source: keep the whole detector
            const double lam = num / den;
#pragma unroll
            for (int e = 0; e < 3; ++e) pt[e] = P.src[e] + lam * dx[e] - P.dc[e];
        }
        const double a = pt[0] * P.ud[0] + pt[1] * P.ud[1] + pt[2] * P.ud[2];
        const double b = pt[0] * P.vd[0] + pt[1] * P.vd[1] + pt[2] * P.vd[2];
        amin = fmin(amin, a);
        amax = fmax(amax, a);
        bmin = fmin(bmin, b);
        bmax = fmax(bmax, b);
    }
    // clamp to the detector before converting (far corners stay in range)
    const double eps = 1e-3;
    u0 = (int)fmin(fmax(0.0, ceil(amin + cu - eps)), (double)g.nu);
    u1 = (int)fmax(fmin((double)(g.nu - 1), floor(amax + cu + eps)), -1.0);
    v0 = (int)fmin(fmax(0.0, ceil(bmin + cv - eps)), (double)g.nv);
    v1 = (int)fmax(fmin((double)(g.nv - 1), floor(bmax + cv + eps)), -1.0);
    return false;
}

// Clip the cell range [cf, cl] of a ray to the cells whose window can hold a
// basis of the brick: over cell c the window's a-range is
// [floor(v_a(c)) - N, floor(v_a(c+1))], v_a(c) = V + (c - c0) r_a (same for
// b).  Conservative by two cells; starting before the first such cell is
// what keeps the brick's values equal to the full march's.
template <int N>
__device__ __forceinline__ void clip_cells_to_brick(const RaySetup &rs, const int (&blo)[3], const int (&bhi)[3],
                                                    int &cf, int &cl)
{
    const float base[2] = {rs.Vah + rs.Val, rs.Vbh + rs.Vbl};
    const float r[2] = {rs.ra, rs.rb}, ir[2] = {rs.inv_ra, rs.inv_rb};
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (r[q] > 0.0f) {
            const float cfl = rs.c0 + (blo[q + 1] - base[q]) * ir[q];
            const float chl = rs.c0 + (bhi[q + 1] + N + 1 - base[q]) * ir[q];
            cf = max(cf, (int)fmaxf(floorf(cfl) - 2.0f, -1e9f));
            cl = min(cl, (int)fminf(ceilf(chl) + 1.0f, 1e9f));
        } else if (!(base[q] + 1.0f > blo[q + 1] && base[q] - (N + 1) < bhi[q + 1])) {
            cl = cf - 1;
        }
    }
}

// vlist: the views to walk (NULL: all views 0 .. nview-1); add: c += the
// brick totals instead of c = them
template <int N>
__global__ void __launch_bounds__(kAdjThreads) k_adjoint_bricks(DevGeom g, const float *__restrict__ y,
                                                                float *__restrict__ c, QuadRule qr, int bx, int by,
                                                                const int *vlist, int nview, int add)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *tot = (double *)smem;                                // kBrickVol FP64 totals
    float *part = (float *)(smem + kBrickVol * sizeof(double));  // kBrickVol partials of a view batch
    __shared__ int win[kViewBatch][3];                           // u0, wu, v0 of each view of the batch
    __shared__ int woff[kViewBatch + 1];                         // prefix sums of the window sizes
    __shared__ int next_item;
    constexpr double W = 0.5 * (N + 1);
    const int bid = blockIdx.x;
    const int b0[3] = {(bid % bx) * kBrick, ((bid / bx) % by) * kBrick, (bid / (bx * by)) * kBrick};
    int bn[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) bn[e] = min(kBrick, g.n[e] - b0[e]);
    for (int i = threadIdx.x; i < kBrickVol; i += kAdjThreads) {
        tot[i] = 0.0;
        part[i] = 0.0f;
    }
    // support box of the brick's bases (world)
    double lo[3], hi[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        lo[e] = g.org[e] + b0[e] - W;
        hi[e] = g.org[e] + b0[e] + bn[e] - 1 + W;
    }
    const GridBox gb = grid_of(g);
    const int lstride[3] = {1, kBrick, kBrick * kBrick};
    bool ok = true;
    __shared__ int vk[kViewBatch];
    for (int k0 = 0; k0 < nview; k0 += kViewBatch) {
        const int nb = min(kViewBatch, nview - k0);
        if (threadIdx.x < nb) {
            const int kv = vlist ? vlist[k0 + threadIdx.x] : k0 + threadIdx.x;
            vk[threadIdx.x] = kv;
            int u0, u1, v0, v1;
            if (pixel_window(g, kv, lo, hi, u0, u1, v0, v1)) {
                u0 = 0;
                u1 = g.nu - 1;
                v0 = 0;
                v1 = g.nv - 1;
            }
            const int wu = u1 - u0 + 1, wv = v1 - v0 + 1;
            win[threadIdx.x][0] = u0;
            win[threadIdx.x][1] = wu > 0 ? wu : 0;
            win[threadIdx.x][2] = v0;
            woff[threadIdx.x + 1] = (wu > 0 && wv > 0) ? wu * wv : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            woff[0] = 0;
            for (int t = 1; t <= nb; ++t) woff[t] += woff[t - 1];
            next_item = 0;
        }
        __syncthreads();
        const int total = woff[nb];
        // rays are taken one at a time from a shared counter: their costs
        // differ a lot (a ray may cross one slab of the brick or sixteen)
        for (int item = atomicAdd(&next_item, 1); item < total; item = atomicAdd(&next_item, 1)) {
            int t = 0;
            while (item >= woff[t + 1]) ++t;
            const int p = item - woff[t];
            const int iu = win[t][0] + p % win[t][1], iv = win[t][2] + p / win[t][1];
            const int k = vk[t];
            const float yr = __ldg(y + ((long long)k * g.nv + iv) * g.nu + iu);
            if (yr == 0.0f) continue;
            RaySetup rs;
            if (!view_setup<N>(g, gb, k, iu, iv, rs)) continue;
            // brick bounds in the ray's mirrored (d, a, b) coordinates
            int blo[3], bhi[3], L[3], Loff = 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int e = rs.ax[q];
                const int r0 = b0[e], r1 = b0[e] + bn[e] - 1;
                blo[q] = rs.sg[q] > 0 ? r0 : -r1;
                bhi[q] = rs.sg[q] > 0 ? r1 : -r0;
                L[q] = rs.sg[q] * lstride[e];
                Loff -= b0[e] * lstride[e];
            }
            // a brick basis l_d is live in cells l_d .. l_d + N
            int cf = max(rs.c0, blo[0]), cl = min(rs.c1, bhi[0] + N);
            clip_cells_to_brick<N>(rs, blo, bhi, cf, cl);
            if (cf > cl) continue;
            BrickSink sk;
            sk.part = part;
            sk.S0 = L[0];
            sk.S1 = L[1];
            sk.S2 = L[2];
            sk.off = (unsigned)Loff;
            sk.bx = make_box(blo, bhi);
            sk.yv = yr * rs.inv_wd;
            ok &= march_kind<N>(g.kind, rs, cf, cl, qr, sk);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kBrickVol; i += kAdjThreads) {
            tot[i] += (double)part[i];
            part[i] = 0.0f;
        }
        __syncthreads();
    }
    if (!ok) atomicOr(g.err, 1);
    for (int i = threadIdx.x; i < kBrickVol; i += kAdjThreads) {
        const int lx = i % kBrick, ly = (i / kBrick) % kBrick, lz = i / (kBrick * kBrick);
        if (lx < bn[0] && ly < bn[1] && lz < bn[2]) {
            float &dst = c[((long long)(b0[2] + lz) * g.n[1] + (b0[1] + ly)) * g.n[0] + (b0[0] + lx)];
            dst = add ? (float)((double)dst + tot[i]) : (float)tot[i];
        }
    }
}

constexpr size_t kAdjSmem = kBrickVol * (sizeof(double) + sizeof(float));

// Batched scatter: acc += c (FP64 total of the batches), and c = acc at the
// end.  Grid-strided, coalesced.
__global__ void k_acc_add(long long n, double *__restrict__ acc, const float *__restrict__ c)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc[i] += (double)c[i];
}

__global__ void k_acc_store(long long n, const double *__restrict__ acc, float *__restrict__ c)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) c[i] = (float)acc[i];
}

}  // namespace spl

using namespace spl;

static spl_status launch_status(const char *what)
{
    return cuda_check(cudaGetLastError(), what);
}

// Launch `launch(chunk, n)` for the parallel views view_order[v0 .. v0+count)
// in chunks of at most `per` (<= kViewChunk) views, each with its views'
// constants.
template <class F>
static void for_view_chunks(const spl_geometry *g, int v0, int count, F launch, int per = kViewChunk)
{
    static thread_local ViewChunk ch;
    for (int s = 0; s < count; s += per) {
        const int n = count - s < per ? count - s : per;
        memcpy(ch.v, g->vconst + v0 + s, (size_t)n * sizeof(ViewConst));
        launch(ch, n);
    }
}

static unsigned stream_grid(long long n)
{
    const long long b = (n + 255) / 256, cap = 8LL * sm_count();
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// Parallel geometries: the separable group through the plane matrices
// (when used), the other flat views with the flat kernel, the rest with the
// general one.  Returns the first view_order index the flat kernel takes.
// The plane matrices are built by spl_prepare only: unbuilt is an error
// (SPL_ERR_STATE), unavailable (their allocation failed) walks the views.
static int plane_views(const spl_geometry *g, const spl_basis_desc *b, spl_status *err)
{
    *err = SPL_OK;
    if (b->separable == SPL_SEP_OFF || b->mode == SPL_FP_MLP || b->mode == SPL_FP_TABLE || !g->plane) return 0;
    const int state = plane_state(g, b->degree);
    if (state == 0) {
        *err = fail(SPL_ERR_STATE, "plane matrices of degree %d not built: call spl_prepare first", b->degree);
        return 0;
    }
    return state == 1 ? g->dev.n_sep : 0;
}

template <int N, bool DIRECT>
static spl_status forward_quad_t(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y,
                                 cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    const QuadRule qr = quad_rule(N);
    const int kahan = b->kahan;
    if (dg.n_rays == 0) return SPL_OK;
    if (dg.kind == SPL_RAYS) {
        const long long blocks = (dg.n_rays + 127) / 128;
        k_forward_rays<N, DIRECT><<<(unsigned)blocks, 128, 0, st>>>(dg, c, y, qr, kahan);
    } else if (dg.kind == SPL_PARALLEL) {
        spl_status s;
        const int v0 = plane_views(g, b, &s);
        if (s != SPL_OK) return s;
        // the plane path (memory-latency bound) runs beside the march of the
        // other views (arithmetic bound) when both have work: the two write
        // disjoint rows of y
        const bool overlap = v0 > 0 && v0 < dg.n_views && g->plane->side;
        if (v0 > 0) {
            cudaStream_t ps = st;
            if (overlap) {
                s = cuda_check(cudaEventRecord(g->plane->fork, st), "fork record");
                if (s == SPL_OK) s = cuda_check(cudaStreamWaitEvent(g->plane->side, g->plane->fork, 0), "fork wait");
                if (s != SPL_OK) return s;
                ps = g->plane->side;
            }
            s = plane_forward(g, N, kahan, c, y, ps);
            if (overlap) {
                const spl_status sj = cuda_check(cudaEventRecord(g->plane->join, ps), "join record");
                if (s != SPL_OK || sj != SPL_OK) {
                    // join the side stream before returning the error, so the
                    // caller's stream (or its graph capture) never leaves it
                    // unjoined
                    if (sj == SPL_OK) cudaStreamWaitEvent(st, g->plane->join, 0);
                    return s != SPL_OK ? s : sj;
                }
            }
            if (s != SPL_OK) return s;
        }
        const unsigned gx = (dg.nu + 15) / 16, gy = (dg.nv + 7) / 8;
        for_view_chunks(g, v0, dg.n_flat - v0, [&](const ViewChunk &ch, int n) {
            k_forward_pviews<N, VM_FLAT, false><<<dim3(gx, gy, n), 128, 0, st>>>(dg, c, y, qr, kahan, ch);
        });
        for_view_chunks(g, dg.n_flat, dg.n_views - dg.n_flat, [&](const ViewChunk &ch, int n) {
            k_forward_pviews<N, VM_GENERAL, DIRECT><<<dim3(gx, gy, n), 128, 0, st>>>(dg, c, y, qr, kahan, ch);
        });
        if (overlap) {
            s = cuda_check(cudaStreamWaitEvent(st, g->plane->join, 0), "join wait");
            if (s != SPL_OK) return s;
        }
    } else {
        dim3 grid((dg.nu + 15) / 16, (dg.nv + 7) / 8, dg.n_views);
        k_forward_views<N, DIRECT><<<grid, 128, 0, st>>>(dg, c, y, qr, kahan);
    }
    return launch_status("forward launch");
}

template <int N>
static spl_status forward_quad(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st)
{
    return b->mode == SPL_FP_DIRECT ? forward_quad_t<N, true>(g, b, c, y, st) : forward_quad_t<N, false>(g, b, c, y, st);
}

template <int N>
static spl_status adjoint_quad(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    const QuadRule qr = quad_rule(N);
    const int form = b->adjoint;
    const long long nc = (long long)dg.n[0] * dg.n[1] * dg.n[2];
    spl_status s = SPL_OK;
    int v0 = 0;
    if (dg.kind == SPL_PARALLEL) {
        v0 = plane_views(g, b, &s);
        if (s != SPL_OK) return s;
    }
    // With the scatter form the plane path's gather (T, memory-latency
    // bound) runs on the geometry's side stream beside the march's scatter
    // into the cleared c (arithmetic bound); after the join, T's
    // contribution is added to c.  Otherwise the plane path writes every
    // coefficient first and the other views add.
    const bool overlap = dg.kind == SPL_PARALLEL && dg.n_rays > 0 && v0 > 0 && v0 < dg.n_views && form != SPL_ADJ_GATHER &&
                         g->plane->side;
    if (overlap) {
        s = cuda_check(cudaEventRecord(g->plane->fork, st), "fork record");
        if (s == SPL_OK) s = cuda_check(cudaStreamWaitEvent(g->plane->side, g->plane->fork, 0), "fork wait");
        if (s != SPL_OK) return s;
        s = plane_adjoint_t(g, N, y, g->plane->side);
        spl_status sj = cuda_check(cudaEventRecord(g->plane->join, g->plane->side), "join record");
        if (s == SPL_OK) s = sj;
        if (s == SPL_OK) s = cuda_check(cudaMemsetAsync(c, 0, nc * sizeof(float), st), "adjoint clear");
        if (s != SPL_OK) {
            // join the side stream before returning the error
            if (sj == SPL_OK) cudaStreamWaitEvent(st, g->plane->join, 0);
            return s;
        }
    } else if (v0 > 0) {
        s = plane_adjoint(g, N, y, c, st);
        if (s != SPL_OK) return s;
    } else if (dg.kind == SPL_RAYS || form != SPL_ADJ_GATHER) {
        s = cuda_check(cudaMemsetAsync(c, 0, nc * sizeof(float), st), "adjoint clear");
        if (s != SPL_OK) return s;
    }
    if (dg.n_rays == 0) return SPL_OK;
    // The scatter adds y_r * F_l with FP32 atomics.  A coefficient of a
    // large geometry receives tens of thousands of them (512^3 helical:
    // ~4e4), and an FP32 running sum of that many terms loses ~1e-5 of its
    // value; so a geometry with more than one batch of views (rays) scatters
    // each batch into the cleared c and adds the batch to an FP64 total
    // (its scratch, acc64, is allocated with the geometry), which is
    // rounded to c at the end.  Each batch's FP32 sum has ~1/B of the terms
    // and of the magnitude, so its rounding error is ~1/B of the whole.
    const bool batched = g->acc64 != nullptr;
    auto begin_batch = [&]() -> spl_status {
        if (!batched) return SPL_OK;
        return cuda_check(cudaMemsetAsync(c, 0, nc * sizeof(float), st), "adjoint batch clear");
    };
    auto end_batch = [&]() {
        if (batched) k_acc_add<<<stream_grid(nc), 256, 0, st>>>(nc, g->acc64, c);
    };
    if (batched && form != SPL_ADJ_GATHER) {
        s = cuda_check(cudaMemsetAsync(g->acc64, 0, nc * sizeof(double), st), "adjoint accumulator clear");
        if (s != SPL_OK) return s;
        // the plane path already wrote its part into c (no side stream):
        // it enters the total first
        if (v0 > 0 && !overlap) end_batch();
    }
    // the b-fast layouts (see b_fast_target), four shifted copies each:
    // cleared before and folded into c after each launch that reduces into
    // them
    const long long nx = dg.n[0], ny = dg.n[1], nz = dg.n[2], cs = (long long)dg.lay_cs;
    auto lay_clear = [&]() -> spl_status {
        spl_status e = SPL_OK;
        for (int L = 0; L < 3 && e == SPL_OK; ++L)
            e = cuda_check(cudaMemsetAsync(g->lay[L], 0, 4 * dg.lay_cs * sizeof(float), st), "adjoint layout clear");
        return e;
    };
    auto lay_fold = [&]() {
        k_fold_copies<<<stream_grid(nc), 256, 0, st>>>(c, g->lay[0], nc, cs);
        k_fold_copies_transpose<<<dim3((unsigned)((nx + 31) / 32), (unsigned)((ny + 31) / 32),
                                       (unsigned)(nz < 65535 ? nz : 65535)),
                                  256, 0, st>>>(c, g->lay[1], nx, ny, nz, cs);
        k_fold_copies_transpose<<<dim3((unsigned)((nx * ny + 31) / 32), (unsigned)((nz + 31) / 32), 1), 256, 0, st>>>(
            c, g->lay[2], nx * ny, nz, 1, cs);
    };
    if (dg.kind == SPL_RAYS) {
        for (long long r0 = 0; r0 < dg.n_rays; r0 += kAdjBatchRays) {
            const long long r1 = r0 + kAdjBatchRays < dg.n_rays ? r0 + kAdjBatchRays : dg.n_rays;
            if ((s = begin_batch()) != SPL_OK || (s = lay_clear()) != SPL_OK) return s;
            k_adjoint_rays<N><<<(unsigned)((r1 - r0 + 127) / 128), 128, 0, st>>>(dg, y, g->lay[0], g->lay[1],
                                                                                  g->lay[2], qr, r0, r1);
            lay_fold();
            end_batch();
        }
        if (batched) k_acc_store<<<stream_grid(nc), 256, 0, st>>>(nc, g->acc64, c);
        return launch_status("adjoint launch");
    }
    if (form != SPL_ADJ_GATHER) {
        const unsigned gx = (dg.nu + 15) / 16, gy = (dg.nv + 7) / 8;
        const int per = batched ? kAdjBatchViews : kViewChunk;
        if (dg.kind == SPL_PARALLEL) {
            for_view_chunks(g, v0, dg.n_flat - v0, [&](const ViewChunk &ch, int n) {
                if (s == SPL_OK) s = begin_batch();
                k_adjoint_pviews_scatter<N, VM_FLAT><<<dim3(gx, gy, n), 128, 0, st>>>(dg, y, c, nullptr, nullptr,
                                                                                    nullptr, qr, ch);
                end_batch();
            }, per);
            for_view_chunks(g, dg.n_flat, dg.n_views - dg.n_flat, [&](const ViewChunk &ch, int n) {
                if (s == SPL_OK) s = begin_batch();
                if (s == SPL_OK) s = lay_clear();
                k_adjoint_pviews_scatter<N, VM_GENERAL><<<dim3(gx, gy, n), 128, 0, st>>>(dg, y, c, g->lay[0], g->lay[1],
                                                                                       g->lay[2], qr, ch);
                lay_fold();
                end_batch();
            }, per);
            if (batched) k_acc_store<<<stream_grid(nc), 256, 0, st>>>(nc, g->acc64, c);
            if (overlap) {
                const spl_status sj = cuda_check(cudaStreamWaitEvent(st, g->plane->join, 0), "join wait");
                if (s == SPL_OK) s = sj;
                if (s == SPL_OK) s = plane_adjoint_add(g, N, c, st);
            }
            if (s != SPL_OK) return s;
        } else {
            const int per_launch = batched ? kAdjBatchViews : dg.n_views;
            for (int k0 = 0; k0 < dg.n_views; k0 += per_launch) {
                const int nview = dg.n_views - k0 < per_launch ? dg.n_views - k0 : per_launch;
                if ((s = begin_batch()) != SPL_OK || (s = lay_clear()) != SPL_OK) return s;
                k_adjoint_views_scatter<N><<<dim3(gx, gy, nview), 128, 0, st>>>(dg, y, g->lay[0], g->lay[1], g->lay[2],
                                                                                 qr, k0);
                lay_fold();
                end_batch();
            }
            if (batched) k_acc_store<<<stream_grid(nc), 256, 0, st>>>(nc, g->acc64, c);
        }
        return launch_status("adjoint launch");
    }
    s = smem_attr_once((const void *)k_adjoint_bricks<N>, (int)kAdjSmem, "adjoint smem attribute");
    if (s != SPL_OK) return s;
    const int bx = (dg.n[0] + kBrick - 1) / kBrick, by = (dg.n[1] + kBrick - 1) / kBrick,
              bz = (dg.n[2] + kBrick - 1) / kBrick;
    // bricks over the views the plane path did not take (all of them
    // without it); with the plane path they add to its result
    const int *vlist = v0 > 0 ? dg.view_order + v0 : nullptr;
    const int nview = dg.n_views - v0;
    k_adjoint_bricks<N><<<bx * by * bz, kAdjThreads, kAdjSmem, st>>>(dg, y, c, qr, bx, by, vlist, nview, v0 > 0 ? 1 : 0);
    return launch_status("adjoint launch");
}

template <int N>
static spl_status count_pairs(const spl_geometry *g, unsigned long long *count, cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    const QuadRule qr = quad_rule(N);
    if (dg.n_rays == 0) return SPL_OK;
    spl_status s = count_exact(g, N, count, nullptr, st);
    if (s != SPL_OK) return s;
    if (dg.kind == SPL_RAYS) {
        const long long blocks = (dg.n_rays + 127) / 128;
        k_count_rays<N><<<(unsigned)blocks, 128, 0, st>>>(dg, count, qr);
    } else {
        dim3 grid((dg.nu + 15) / 16, (dg.nv + 7) / 8, dg.n_views);
        k_count_views<N><<<grid, 128, 0, st>>>(dg, count, qr);
    }
    return launch_status("count launch");
}

// c: coefficient array (never empty); y: projection array (may be empty, and
// then NULL)
static spl_status check_call(const spl_geometry *g, const spl_basis_desc *b, const void *c, const void *y)
{
    clear_error();
    if (!g) return fail(SPL_ERR_ARG, "geometry is NULL");
    spl_status s = check_basis(b);
    if (s != SPL_OK) return s;
    if (!c) return fail(SPL_ERR_ARG, "coefficient pointer is NULL");
    if (!y && g->dev.n_rays > 0) return fail(SPL_ERR_ARG, "projection pointer is NULL");
    if (b->mode == SPL_FP_MLP) {
        if (spl_mlp_degree(b->mlp) != b->degree)
            return fail(SPL_ERR_ARG, "MLP degree %d does not match basis degree %d", spl_mlp_degree(b->mlp), b->degree);
        if (g->dev.kind == SPL_RAYS) return fail(SPL_ERR_UNSUPPORTED, "MLP footprint needs a view geometry");
    }
    return SPL_OK;
}

#define SPL_DISPATCH(deg, fn, ...)                                                                                   \
    switch (deg) {                                                                                                   \
    case 0: return fn<0>(__VA_ARGS__);                                                                               \
    case 1: return fn<1>(__VA_ARGS__);                                                                               \
    case 2: return fn<2>(__VA_ARGS__);                                                                               \
    default: return fn<3>(__VA_ARGS__);                                                                              \
    }

extern "C" spl_status spl_forward(const spl_geometry *g, const spl_basis_desc *b, const float *c_dev, float *y_dev,
                                  void *stream)
{
    spl_status s = check_call(g, b, c_dev, y_dev);
    if (s != SPL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->mode == SPL_FP_MLP) return spl::forward_mlp(g, b, c_dev, y_dev, st);
    if (b->mode == SPL_FP_TABLE) return spl::table_forward(g, b, c_dev, y_dev, st);
    SPL_DISPATCH(b->degree, forward_quad, g, b, c_dev, y_dev, st)
}

extern "C" spl_status spl_adjoint(const spl_geometry *g, const spl_basis_desc *b, const float *y_dev, float *c_dev,
                                  void *stream)
{
    spl_status s = check_call(g, b, c_dev, y_dev);
    if (s != SPL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (b->mode == SPL_FP_MLP) return spl::adjoint_mlp(g, b, y_dev, c_dev, st);
    if (b->mode == SPL_FP_TABLE) return spl::table_adjoint(g, b, y_dev, c_dev, st);
    if (b->adjoint != SPL_ADJ_AUTO && b->adjoint != SPL_ADJ_GATHER && b->adjoint != SPL_ADJ_SCATTER)
        return fail(SPL_ERR_ARG, "unknown adjoint form %d", b->adjoint);
    SPL_DISPATCH(b->degree, adjoint_quad, g, b, y_dev, c_dev, st)
}

extern "C" spl_status spl_count_pairs(const spl_geometry *g, int degree, unsigned long long *count_dev, void *stream)
{
    clear_error();
    if (!g || !count_dev) return fail(SPL_ERR_ARG, "NULL argument");
    if (degree < 0 || degree > 3) return fail(SPL_ERR_ARG, "degree %d not in 0..3", degree);
    SPL_DISPATCH(degree, count_pairs, g, count_dev, (cudaStream_t)stream)
}
