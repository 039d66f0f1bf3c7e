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

// The frame of the features in the caller's coordinates: with G the
// signed permutation above (chamber direction Gw) and the chamber frame
// u_c = normalize(e1 x Gw), v_c = u_c x Gw, returns u = G^T u_c and
// v = G^T v_c, so that <Gp, u_c> = <p, u> and <Gp, v_c> = <p, v>: the last
// two features are <p, u> sqrt3/W and <p, v> sqrt3/W.  u and v are an
// orthonormal basis of the plane perpendicular to w, and
// v = det(G) (u x w).  FP64.
__host__ __device__ inline void canonical_frame(const double (&w_in)[3], double (&u_out)[3], double (&v_out)[3])
{
    double w[3];
    int idx[3], sg[3];
    for (int e = 0; e < 3; ++e) {
        sg[e] = w_in[e] < 0.0 ? -1 : 1;
        w[e] = w_in[e] < 0.0 ? -w_in[e] : w_in[e];
        idx[e] = e;
    }
    // the same stable ascending sort as canonical_features, tracking which
    // axis lands in each chamber position
    for (int i = 1; i < 3; ++i)
        for (int j = i; j > 0 && w[j - 1] > w[j]; --j) {
            const double t = w[j];
            w[j] = w[j - 1];
            w[j - 1] = t;
            const int k = idx[j];
            idx[j] = idx[j - 1];
            idx[j - 1] = k;
        }
    const double nr = sqrt(w[1] * w[1] + w[2] * w[2]);
    const double u[3] = {0.0, -w[2] / nr, w[1] / nr};
    const double v[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    // chamber component j is sg[idx[j]] times the caller's component idx[j]
    for (int j = 0; j < 3; ++j) {
        u_out[idx[j]] = sg[idx[j]] * u[j];
        v_out[idx[j]] = sg[idx[j]] * v[j];
    }
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
// Evaluation copy of the parameters: the two 64x64 layers as BF16 rows of
// 36 words (32 used; every 16-byte unit of a row is 16-byte aligned, the
// unit the tcgen05 tile set-up copies), the rest as FP32: W1 and W4 holding
// BF16-rounded weights, the biases unrounded.
constexpr int kRowWords = 36;  // 32-bit words per padded W2 / W3 row
struct MlpDev {
    const uint32_t *w23;  // [2][64][36] BF16 pairs: W2 then W3, row = output unit
    const float *f32;     // W1 [64][5], b1 [64], b2 [64], b3 [64], W4 [64], b4 [1]
    const void *tc_img;   // the same network in the tcgen05 tile's operand layout
    int *err;             // device error flag of the network (bit 1: a tensor-core wait gave up)
};
// bits of the device error flags (geometry and MLP): a loop bound was
// reached / a bounded tensor-core completion wait gave up
constexpr int kErrStepCap = 1, kErrTimeout = 2;
constexpr int kF32W1 = 0, kF32B1 = 320, kF32B2 = 384, kF32B3 = 448, kF32W4 = 512, kF32B4 = 576, kF32Size = 577;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
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
