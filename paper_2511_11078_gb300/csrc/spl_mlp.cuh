// spl_mlp.cuh -- learned footprint f_theta (Sec. 2.2, Algorithm 1): shared
// declarations and the canonical input features.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "spl_host.h"

namespace spl {

// f_theta architecture: 5 -> 64 -> 64 -> 64 -> 1, SiLU after each hidden layer
constexpr int kIn = 5;
constexpr int kHid = 64;
constexpr int kParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kHid + 1;  // 8769
// offsets of each layer's W [out][in] and b [out] in the parameter vector
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn;
constexpr int kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid, kOffB4 = kOffW4 + kHid;

// MLP input features of (w, p): signed permutation G mapping w into the
// chamber 0 <= w1 <= w2 <= w3 (phi is invariant under it, so
// Pphi(Gw, Gp) = Pphi(w, p)), frame u = normalize(e1 x Gw), v = u x Gw, and
// (Gw1, Gw2, Gw3, <Gp,u> sqrt3/W, <Gp,v> sqrt3/W): the sampling disc of
// radius sqrt3 W maps to radius 3, wide enough in feature space for the
// footprint bump to be learned quickly.  FP64.
__host__ __device__ inline void canonical_features(int degree, const double (&w_in)[3], const double (&p_in)[3],
                                                   double (&f)[5])
{
    const double W = 0.5 * (degree + 1);
    double w[3], p[3];
    for (int e = 0; e < 3; ++e) {
        const bool neg = w_in[e] < 0.0;
        w[e] = neg ? -w_in[e] : w_in[e];
        p[e] = neg ? -p_in[e] : p_in[e];
    }
    // stable ascending sort of three (w, p) pairs by w
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && w[j - 1] > w[j]; --j) {
            double t = w[j];
            w[j] = w[j - 1];
            w[j - 1] = t;
            t = p[j];
            p[j] = p[j - 1];
            p[j - 1] = t;
        }
    const double nr = sqrt(w[1] * w[1] + w[2] * w[2]);
    const double u[3] = {0.0, -w[2] / nr, w[1] / nr};
    const double v[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    const double sc = sqrt(3.0) / W;
    f[0] = w[0];
    f[1] = w[1];
    f[2] = w[2];
    f[3] = (p[0] * u[0] + p[1] * u[1] + p[2] * u[2]) * sc;
    f[4] = (p[0] * v[0] + p[1] * v[1] + p[2] * v[2]) * sc;
}

// The same features in FP32 (the library's FP64 units are scarce on GB300;
// the features are FP32 values either way).  Same flip, stable sort and frame.
__device__ __forceinline__ void canonical_features_f32(int degree, const float (&w_in)[3], const float (&p_in)[3],
                                                       float (&f)[5])
{
    const float W = 0.5f * (degree + 1);
    float w[3], p[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const bool neg = w_in[e] < 0.0f;
        w[e] = neg ? -w_in[e] : w_in[e];
        p[e] = neg ? -p_in[e] : p_in[e];
    }
#pragma unroll
    for (int i = 1; i < 3; ++i)
#pragma unroll
        for (int j = i; j > 0; --j) {
            const bool sw = w[j - 1] > w[j];
            const float a = w[j - 1], b = w[j], pa = p[j - 1], pb = p[j];
            w[j - 1] = sw ? b : a;
            w[j] = sw ? a : b;
            p[j - 1] = sw ? pb : pa;
            p[j] = sw ? pa : pb;
        }
    const float inr = rsqrtf(w[1] * w[1] + w[2] * w[2]);
    const float u1 = -w[2] * inr, u2 = w[1] * inr;  // u = (0, u1, u2)
    const float v0 = u1 * w[2] - u2 * w[1], v1 = u2 * w[0], v2 = -u1 * w[0];
    const float sc = 1.7320508075688772f / W;
    f[0] = w[0];
    f[1] = w[1];
    f[2] = w[2];
    f[3] = (p[1] * u1 + p[2] * u2) * sc;
    f[4] = (p[0] * v0 + p[1] * v1 + p[2] * v2) * sc;
}

// ---------------------------------------------------------------- device weights
// Evaluation copy of the parameters: the two 64x64 layers as BF16 with a
// padded row stride (72 BF16 = 36 words: the B-fragment loads of a warp hit
// 32 distinct banks), the rest as FP32 holding BF16-rounded weights.
constexpr int kRowWords = 36;  // 32-bit words per padded W2 / W3 row
struct MlpDev {
    const uint32_t *w23;  // [2][64][36] BF16 pairs: W2 then W3, row = output unit
    const float *f32;     // W1 [64][5], b1 [64], b2 [64], b3 [64], W4 [64], b4 [1]
};
constexpr int kF32W1 = 0, kF32B1 = 320, kF32B2 = 384, kF32B3 = 448, kF32W4 = 512, kF32B4 = 576, kF32Size = 577;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}
// the same for values that are BF16 numbers already (no rounding happens)
__device__ __forceinline__ uint32_t pack_bf16_exact(float lo, float hi) { return pack_bf16(lo, hi); }

// Shared-memory copy of the weights, laid out as per-lane mma.sync B
// fragments (m16n8k16, lane = 4 g + t) so that a lane fetches the
// fragments of two k-steps with one 16-byte load, bank-conflict free:
//   w2f / w3f [nt][h][lane] = (b0, b1 of k-step 2h, b0, b1 of k-step 2h+1),
//     b0 = W[8 nt + g][16 kt + 2t, +1], b1 = W[8 nt + g][16 kt + 2t + 8, +9];
//   w1f [p][lane] = (b0, b1 of n-tile 2p, b0, b1 of n-tile 2p+1) for the
//     layer-1 operand below.
struct MlpSmem {
    uint4 w1f[4][32];
    uint4 w2f[8][2][32];
    uint4 w3f[8][2][32];
    float f32[kF32Size + 3];
};

// Layer 1 as one k-step of BF16 MMAs.  A feature x is split into three
// BF16 parts x = hi + mid + lo + r: hi and mid truncate the mantissa to
// 8 bits (the differences are exact in FP32), lo rounds the remainder to
// nearest, so |r| <= 2^-23 |x|.  The 16 columns of the A operand are, for
// the lane quad t = 0..3 holding columns 2t, 2t+1, 2t+8, 2t+9:
//   (hi(x_t), mid(x_t), lo(x_t), part t of x_4)   (part 3 of x_4 is 0),
// so the B operand repeats W1[:, t] three times and holds W1[:, 4] in the
// fourth slot of quads 0..2.  The products are exact and accumulate in FP32
// on the bias b1, which gives z1 to FP32 accuracy.
__device__ __forceinline__ uint32_t w1_pair(const float *W1, int n, int t, int slot)
{
    const float a = W1[n * 5 + t];
    const float b = slot == 0 ? a : (t < 3 ? W1[n * 5 + 4] : 0.0f);
    return pack_bf16_exact(a, b);
}

__device__ __forceinline__ void mlp_load_smem(const MlpDev &w, MlpSmem &S)
{
    // hidden layers: W[n][k] pairs from the padded global rows
    for (int i = threadIdx.x; i < 2 * 8 * 2 * 32 * 4; i += blockDim.x) {
        const int j = i & 3, lane = (i >> 2) & 31, h = (i >> 7) & 1, nt = (i >> 8) & 7, layer = i >> 11;
        const int g = lane >> 2, t = lane & 3, kt = 2 * h + (j >> 1), which = j & 1;
        const uint32_t v = w.w23[layer * kHid * kRowWords + (8 * nt + g) * kRowWords + 8 * kt + t + 4 * which];
        uint32_t *dst = reinterpret_cast<uint32_t *>(layer == 0 ? &S.w2f[nt][h][lane] : &S.w3f[nt][h][lane]);
        dst[j] = v;
    }
    for (int i = threadIdx.x; i < 4 * 32 * 4; i += blockDim.x) {
        const int j = i & 3, lane = (i >> 2) & 31, p = i >> 7;
        const int g = lane >> 2, t = lane & 3, nt = 2 * p + (j >> 1);
        reinterpret_cast<uint32_t *>(&S.w1f[p][lane])[j] = w1_pair(w.f32 + kF32W1, 8 * nt + g, t, j & 1);
    }
    for (int i = threadIdx.x; i < kF32Size; i += blockDim.x) S.f32[i] = w.f32[i];
}

// SiLU(z) = z / (1 + 2^(-z log2 e)) of two values: packed FP32x2 multiply and
// add, the MUFU base-2 exponential and reciprocal (relative error ~1e-6);
// saturates correctly for large |z| (2^(+big) = inf gives -0, 2^(-big) = 0
// gives z).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 silu2(float2 z)
{
    constexpr float kNegLog2e = -1.4426950408889634f;
    const float2 m = __fmul2_rn(z, make_float2(kNegLog2e, kNegLog2e));
    const float2 d = __fadd2_rn(make_float2(ex2_approx(m.x), ex2_approx(m.y)), make_float2(1.0f, 1.0f));
    return __fmul2_rn(z, make_float2(rcp_approx(d.x), rcp_approx(d.y)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Optional capture of the activations of one 16-row tile (training):
// z1, h1, z2, h2, z3, h3 (FP32; h1, h2 as the BF16-rounded values that
// entered the tensor-core layers), each [rows][64] with row stride 64.
struct MlpSave {
    float *z1, *h1, *z2, *h2, *z3, *h3;
    int row_g, row_g8;  // destination rows of this lane's rows g and g+8 (-1: skip)
};

// The A operand of layer 1 for one row x of the lane (r = 0: row g, r = 1:
// row g+8).
__device__ __forceinline__ void layer1_row(const float (&x)[5], int t, uint32_t &hi_mid, uint32_t &lo_x4)
{
    const float xt = t == 0 ? x[0] : (t == 1 ? x[1] : (t == 2 ? x[2] : x[3]));
    const uint32_t bx = __float_as_uint(xt);
    const float r1 = xt - __uint_as_float(bx & 0xFFFF0000u);
    const uint32_t b1 = __float_as_uint(r1);
    const float r2 = r1 - __uint_as_float(b1 & 0xFFFF0000u);
    const float h4 = __uint_as_float(__float_as_uint(x[4]) & 0xFFFF0000u);
    const float q1 = x[4] - h4;
    const float m4 = __uint_as_float(__float_as_uint(q1) & 0xFFFF0000u);
    const float s4 = t == 0 ? h4 : (t == 1 ? m4 : (t == 2 ? q1 - m4 : 0.0f));
    hi_mid = __byte_perm(bx, b1, 0x7632);  // (hi, mid): the truncated halves
    lo_x4 = pack_bf16(r2, s4);             // (lo, part t of x_4), rounded to nearest
}

// Bias into the accumulators of n-tile nt (columns 8 nt + 2t, +1 of rows
// g and g+8).
__device__ __forceinline__ void bias_init(const float *B, int nt, int t, float (&c)[4])
{
    const float2 b = *reinterpret_cast<const float2 *>(B + 8 * nt + 2 * t);
    c[0] = b.x;
    c[1] = b.y;
    c[2] = b.x;
    c[3] = b.y;
}

// SiLU of a layer's accumulators (z in C, h out in C); SAVE stores z.
template <bool SAVE>
__device__ __forceinline__ void silu_layer(float (&C)[8][4], int t, float *zb, const MlpSave *sv)
{
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + 2 * t;
        if (SAVE) {
            if (sv->row_g >= 0) {
                zb[sv->row_g * 64 + col] = C[nt][0];
                zb[sv->row_g * 64 + col + 1] = C[nt][1];
            }
            if (sv->row_g8 >= 0) {
                zb[sv->row_g8 * 64 + col] = C[nt][2];
                zb[sv->row_g8 * 64 + col + 1] = C[nt][3];
            }
        }
        const float2 h0 = silu2(make_float2(C[nt][0], C[nt][1]));
        const float2 h1 = silu2(make_float2(C[nt][2], C[nt][3]));
        C[nt][0] = h0.x;
        C[nt][1] = h0.y;
        C[nt][2] = h1.x;
        C[nt][3] = h1.y;
    }
}

// Re-pack a layer's output fragments (BF16-rounded) as the A operand of the
// next MMA layer; SAVE stores the rounded values.
template <bool SAVE>
__device__ __forceinline__ void repack(const float (&C)[8][4], int t, uint32_t (&A)[4][4], float *hb, const MlpSave *sv)
{
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        A[kt][0] = pack_bf16(C[2 * kt][0], C[2 * kt][1]);
        A[kt][1] = pack_bf16(C[2 * kt][2], C[2 * kt][3]);
        A[kt][2] = pack_bf16(C[2 * kt + 1][0], C[2 * kt + 1][1]);
        A[kt][3] = pack_bf16(C[2 * kt + 1][2], C[2 * kt + 1][3]);
    }
    if (SAVE) {
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int col = 16 * kt + 2 * t + 8 * half;
                const __nv_bfloat162 ha = *reinterpret_cast<const __nv_bfloat162 *>(&A[kt][2 * half]);
                const __nv_bfloat162 hc = *reinterpret_cast<const __nv_bfloat162 *>(&A[kt][2 * half + 1]);
                if (sv->row_g >= 0) {
                    hb[sv->row_g * 64 + col] = __bfloat162float(ha.x);
                    hb[sv->row_g * 64 + col + 1] = __bfloat162float(ha.y);
                }
                if (sv->row_g8 >= 0) {
                    hb[sv->row_g8 * 64 + col] = __bfloat162float(hc.x);
                    hb[sv->row_g8 * 64 + col + 1] = __bfloat162float(hc.y);
                }
            }
    }
}

// Hidden-to-hidden layer on the tensor cores: C = b + A * W^T for the 16
// rows of the tile, 8 n-tiles x 4 k-steps of m16n8k16 BF16 MMAs (FP32
// accumulate).
__device__ __forceinline__ void mlp_hidden_layer(const uint4 (&Wf)[8][2][32], const float *B, const uint32_t (&A)[4][4],
                                                 int lane, float (&C)[8][4])
{
    const int t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        bias_init(B, nt, t, C[nt]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 f = Wf[nt][h][lane];
            mma_bf16(C[nt], A[2 * h], f.x, f.y);
            mma_bf16(C[nt], A[2 * h + 1], f.z, f.w);
        }
    }
}

// f_theta on one 16-row tile held by a warp (mma.sync fragment layout: lane
// = 4 g + t holds rows g and g+8).  x_g / x_g8: the 5 features of the lane's
// two rows.  Returns the outputs of rows g and g+8 (in every lane of the
// quad).  Layers 1-3 are BF16 MMAs with FP32 accumulation (layer 1 on the
// three-part split of the FP32 features, so it keeps FP32 accuracy); the
// output layer is FP32 on the CUDA cores.
template <bool SAVE>
__device__ __forceinline__ void mlp_tile16(const MlpSmem &S, const float (&x_g)[5], const float (&x_g8)[5],
                                           float &out_g, float &out_g8, const MlpSave *sv = nullptr)
{
    const int lane = threadIdx.x & 31, t = lane & 3;
    float C[8][4];
    uint32_t A[4][4];
    // ---- layer 1 (5 -> 64)
    {
        uint32_t a1[4];
        layer1_row(x_g, t, a1[0], a1[2]);
        layer1_row(x_g8, t, a1[1], a1[3]);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint4 f = S.w1f[p][lane];
            bias_init(S.f32 + kF32B1, 2 * p, t, C[2 * p]);
            bias_init(S.f32 + kF32B1, 2 * p + 1, t, C[2 * p + 1]);
            mma_bf16(C[2 * p], a1, f.x, f.y);
            mma_bf16(C[2 * p + 1], a1, f.z, f.w);
        }
    }
    silu_layer<SAVE>(C, t, SAVE ? sv->z1 : nullptr, sv);
    repack<SAVE>(C, t, A, SAVE ? sv->h1 : nullptr, sv);
    // ---- layers 2 and 3 (64 -> 64)
    mlp_hidden_layer(S.w2f, S.f32 + kF32B2, A, lane, C);
    silu_layer<SAVE>(C, t, SAVE ? sv->z2 : nullptr, sv);
    repack<SAVE>(C, t, A, SAVE ? sv->h2 : nullptr, sv);
    mlp_hidden_layer(S.w3f, S.f32 + kF32B3, A, lane, C);
    silu_layer<SAVE>(C, t, SAVE ? sv->z3 : nullptr, sv);
    // ---- layer 4 (64 -> 1), FP32
    const float *W4 = S.f32 + kF32W4;
    float og = 0.0f, og8 = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float2 w4 = *reinterpret_cast<const float2 *>(W4 + col);
        og = fmaf(C[nt][0], w4.x, fmaf(C[nt][1], w4.y, og));
        og8 = fmaf(C[nt][2], w4.x, fmaf(C[nt][3], w4.y, og8));
        if (SAVE) {
            if (sv->row_g >= 0) {
                sv->h3[sv->row_g * 64 + col] = C[nt][0];
                sv->h3[sv->row_g * 64 + col + 1] = C[nt][1];
            }
            if (sv->row_g8 >= 0) {
                sv->h3[sv->row_g8 * 64 + col] = C[nt][2];
                sv->h3[sv->row_g8 * 64 + col + 1] = C[nt][3];
            }
        }
    }
    og += __shfl_xor_sync(0xffffffffu, og, 1);
    og += __shfl_xor_sync(0xffffffffu, og, 2);
    og8 += __shfl_xor_sync(0xffffffffu, og8, 1);
    og8 += __shfl_xor_sync(0xffffffffu, og8, 2);
    out_g = og + S.f32[kF32B4];
    out_g8 = og8 + S.f32[kF32B4];
}

// Per-ray data of the learned footprint: canonical direction and the
// (u, v) frame restricted to the ray's mirrored transverse axes, so that
// the features of basis l' = (j, la, lb) are
//   (wc1, wc2, wc3, ua Pa + ub Pb, va Pa + vb Pb),  Pa = A_j - la, Pb = B_j - lb.
struct MlpRay {
    float wc[3];
    float ua, ub, va, vb;
};

// The same signed permutation as canonical_features (flip negative
// components, stable ascending sort): position of each world axis in the
// canonical order, and the scaled frame components for the ray's (a, b).
__device__ __forceinline__ void mlp_ray_setup(int degree, const double (&w)[3], const int (&ax)[3], MlpRay &mr)
{
    const double W = 0.5 * (degree + 1);
    double aw[3];
    int ord[3] = {0, 1, 2};
    for (int e = 0; e < 3; ++e) aw[e] = w[e] < 0.0 ? -w[e] : w[e];
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && aw[ord[j - 1]] > aw[ord[j]]; --j) {
            const int tmp = ord[j];
            ord[j] = ord[j - 1];
            ord[j - 1] = tmp;
        }
    const double w0 = aw[ord[0]], w1 = aw[ord[1]], w2 = aw[ord[2]];
    const double nr = sqrt(w1 * w1 + w2 * w2);
    const double u[3] = {0.0, -w2 / nr, w1 / nr};
    const double v[3] = {u[1] * w2 - u[2] * w1, u[2] * w0 - u[0] * w2, u[0] * w1 - u[1] * w0};
    const double sc = sqrt(3.0) / W;
    int pos[3];
    for (int k = 0; k < 3; ++k) pos[ord[k]] = k;
    mr.wc[0] = (float)w0;
    mr.wc[1] = (float)w1;
    mr.wc[2] = (float)w2;
    mr.ua = (float)(sc * u[pos[ax[1]]]);
    mr.ub = (float)(sc * u[pos[ax[2]]]);
    mr.va = (float)(sc * v[pos[ax[1]]]);
    mr.vb = (float)(sc * v[pos[ax[2]]]);
}

spl_status forward_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st);
spl_status adjoint_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st);
spl_status footprint_mlp(const spl_basis_desc *b, long long count, const float *w, const float *p, float *out,
                         cudaStream_t st);
MlpDev mlp_dev(const spl_mlp *m);

}  // namespace spl
