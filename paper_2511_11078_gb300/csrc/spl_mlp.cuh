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

struct MlpSmem {
    uint32_t w2[kHid * kRowWords];
    uint32_t w3[kHid * kRowWords];
    float f32[kF32Size + 3];
};

__device__ __forceinline__ void mlp_load_smem(const MlpDev &w, MlpSmem &S)
{
    for (int i = threadIdx.x; i < kHid * kRowWords; i += blockDim.x) {
        S.w2[i] = w.w23[i];
        S.w3[i] = w.w23[kHid * kRowWords + i];
    }
    for (int i = threadIdx.x; i < kF32Size; i += blockDim.x) S.f32[i] = w.f32[i];
}

// SiLU(z) = z / (1 + exp(-z)) with the fast exponential and division
// (relative error ~1e-6, two MUFU operations); saturates correctly for
// large |z| (exp(-z) = inf gives -0, exp(-z) = 0 gives z).
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
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

// Hidden-to-hidden layer on the tensor cores: C = A * W^T for the 16 rows of
// the tile, 8 n-tiles x 4 k-tiles of m16n8k16 BF16 MMAs (FP32 accumulate).
__device__ __forceinline__ void mlp_hidden_layer(const uint32_t *Ws, const uint32_t (&A)[4][4], int g, int t,
                                                 float (&C)[8][4])
{
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        C[nt][0] = C[nt][1] = C[nt][2] = C[nt][3] = 0.0f;
        const uint32_t *row = Ws + (8 * nt + g) * kRowWords + t;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_bf16(C[nt], A[kt], row[8 * kt], row[8 * kt + 4]);
    }
}

// f_theta on one 16-row tile held by a warp (mma.sync fragment layout: lane
// = 4 g + t holds rows g and g+8).  x_g / x_g8: the 5 features of the lane's
// two rows.  Returns the outputs of rows g and g+8 (in every lane of the
// quad).  Layer 1 and the output layer are FP32 on the CUDA cores; layers 2
// and 3 are BF16 MMAs whose A operands are the previous layer's output
// fragments re-packed in registers.
template <bool SAVE>
__device__ __forceinline__ void mlp_tile16(const MlpSmem &S, const float (&x_g)[5], const float (&x_g8)[5],
                                           float &out_g, float &out_g8, const MlpSave *sv = nullptr)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float *W1 = S.f32 + kF32W1, *B1 = S.f32 + kF32B1;
    // ---- layer 1 (5 -> 64), FP32: the lane's 16 columns of rows g, g+8
    uint32_t A[4][4];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int c0 = 16 * kt + 2 * t + 8 * half;
            float z[2][2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int col = c0 + cc;
                float za = B1[col], zb = B1[col];
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    za = fmaf(W1[col * 5 + i], x_g[i], za);
                    zb = fmaf(W1[col * 5 + i], x_g8[i], zb);
                }
                z[0][cc] = za;
                z[1][cc] = zb;
            }
            const float h00 = silu_f(z[0][0]), h01 = silu_f(z[0][1]), h10 = silu_f(z[1][0]), h11 = silu_f(z[1][1]);
            A[kt][2 * half] = pack_bf16(h00, h01);
            A[kt][2 * half + 1] = pack_bf16(h10, h11);
            if (SAVE) {
                if (sv->row_g >= 0) {
                    float *zr = sv->z1 + sv->row_g * 64 + c0, *hr = sv->h1 + sv->row_g * 64 + c0;
                    const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&A[kt][2 * half]);
                    zr[0] = z[0][0];
                    zr[1] = z[0][1];
                    hr[0] = __bfloat162float(hb.x);
                    hr[1] = __bfloat162float(hb.y);
                }
                if (sv->row_g8 >= 0) {
                    float *zr = sv->z1 + sv->row_g8 * 64 + c0, *hr = sv->h1 + sv->row_g8 * 64 + c0;
                    const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&A[kt][2 * half + 1]);
                    zr[0] = z[1][0];
                    zr[1] = z[1][1];
                    hr[0] = __bfloat162float(hb.x);
                    hr[1] = __bfloat162float(hb.y);
                }
            }
        }
    }
    // ---- layers 2 and 3 (64 -> 64), BF16 tensor cores
    float C[8][4];
#pragma unroll
    for (int layer = 0; layer < 2; ++layer) {
        const uint32_t *Ws = layer == 0 ? S.w2 : S.w3;
        const float *Bb = S.f32 + (layer == 0 ? kF32B2 : kF32B3);
        mlp_hidden_layer(Ws, A, g, t, C);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int col = 8 * nt + 2 * t;
            float z[4] = {C[nt][0] + Bb[col], C[nt][1] + Bb[col + 1], C[nt][2] + Bb[col], C[nt][3] + Bb[col + 1]};
#pragma unroll
            for (int q = 0; q < 4; ++q) C[nt][q] = silu_f(z[q]);
            if (SAVE) {
                float *zb = layer == 0 ? sv->z2 : sv->z3;
                if (sv->row_g >= 0) {
                    zb[sv->row_g * 64 + col] = z[0];
                    zb[sv->row_g * 64 + col + 1] = z[1];
                }
                if (sv->row_g8 >= 0) {
                    zb[sv->row_g8 * 64 + col] = z[2];
                    zb[sv->row_g8 * 64 + col + 1] = z[3];
                }
            }
        }
        if (layer == 0) {
            // re-pack the output fragments as the A operand of layer 3
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
                        const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162 *>(&A[kt][2 * half + 1]);
                        if (sv->row_g >= 0) {
                            sv->h2[sv->row_g * 64 + col] = __bfloat162float(ha.x);
                            sv->h2[sv->row_g * 64 + col + 1] = __bfloat162float(ha.y);
                        }
                        if (sv->row_g8 >= 0) {
                            sv->h2[sv->row_g8 * 64 + col] = __bfloat162float(hb.x);
                            sv->h2[sv->row_g8 * 64 + col + 1] = __bfloat162float(hb.y);
                        }
                    }
            }
        }
    }
    // ---- layer 4 (64 -> 1), FP32
    const float *W4 = S.f32 + kF32W4;
    float og = 0.0f, og8 = 0.0f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int col = 8 * nt + 2 * t;
        og = fmaf(C[nt][0], W4[col], fmaf(C[nt][1], W4[col + 1], og));
        og8 = fmaf(C[nt][2], W4[col], fmaf(C[nt][3], W4[col + 1], og8));
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
