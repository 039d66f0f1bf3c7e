// mlp.cu -- the learned footprint f_theta (Sec. 2.2) and its training
// (Algorithm 1): parameters, BF16 evaluation copy, batched evaluation on the
// tensor cores, the MLP footprint of spl_footprint, gradients of the L2
// loss and Adam.
//
// Training step (all kernels here, one stream, no host sync):
//   k_train_forward  -- the inference tile (tcgen05 BF16 MMAs) on the batch,
//                       saving pre-activations and the activations that
//                       entered each layer;
//   k_train_backward -- one thread per row: dL/dz of every layer (FP32, the
//                       BF16 roundings passed straight through);
//   k_train_wgrad    -- per batch chunk, dL/dW = sum_b dz_b x h_b^T and
//                       dL/db (FP32), into fixed partial slots;
//   k_train_reduce   -- adds the chunk partials in a fixed order (deterministic)
//                       and the loss;
//   k_adam           -- Adam on the FP32 master copy, then k_prep refreshes
//                       the BF16 evaluation copy.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "spl_mlp.cuh"
#include "spl_tc.cuh"

namespace spl {

constexpr int kChunkRows = 64;     // rows per weight-gradient partial
constexpr int kWgThreads = 256;

}  // namespace spl

struct spl_mlp {
    int degree;
    int max_batch;
    int device;
    int step;
    unsigned long long seed;  // seed of the initial parameters
    float *master;    // [kParams] FP32 master parameters
    float *adam_m;    // [kParams]
    float *adam_v;    // [kParams]
    float *grad;      // [kParams]
    uint32_t *w23;    // evaluation copy, BF16 hidden layers
    float *f32;       // evaluation copy, FP32 first/last layers and biases
    void *tc_img;     // evaluation copy in the tcgen05 tile's operand layout
    float *act;       // [6][max_batch][64] z1 h1 z2 h2 z3 h3
    float *out;       // [max_batch] outputs
    float *dz;        // [3][max_batch][64] dz1 dz2 dz3
    float *dz4;       // [max_batch]
    float *part;      // [chunks][kParams + 1] weight-gradient (and loss) partials
    double *loss_part;  // [max_batch / 128 + 1] per-block loss partials
    int *err;         // device error flag (kErrTimeout: a tensor-core wait gave up)
    void *block;      // single device allocation holding all of the above
};

namespace spl {

MlpDev mlp_dev(const spl_mlp *m)
{
    MlpDev d;
    d.w23 = m->w23;
    d.f32 = m->f32;
    d.tc_img = m->tc_img;
    d.err = m->err;
    return d;
}

// ---------------------------------------------------------------- evaluation copy
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void k_prep(const float *__restrict__ P, uint32_t *__restrict__ w23, float *__restrict__ f32,
                       TcMlpImage *img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // the tcgen05 tile's image of the same roundings
    tc_mlp_image(P, *img, i, gridDim.x * blockDim.x);
    // hidden layers: rows of W2 / W3 as BF16 pairs, padded stride
    if (i < 2 * kHid * kRowWords) {
        const int layer = i / (kHid * kRowWords), rem = i % (kHid * kRowWords);
        const int row = rem / kRowWords, w = rem % kRowWords;
        const float *W = P + (layer == 0 ? kOffW2 : kOffW3);
        uint32_t v = 0;
        if (w < kHid / 2) v = pack_bf16(W[row * kHid + 2 * w], W[row * kHid + 2 * w + 1]);
        w23[i] = v;
    }
    if (i < kF32Size) {
        float v;
        if (i < kF32B1) v = bf16r(P[kOffW1 + i]);
        else if (i < kF32B2) v = P[kOffB1 + (i - kF32B1)];
        else if (i < kF32B3) v = P[kOffB2 + (i - kF32B2)];
        else if (i < kF32W4) v = P[kOffB3 + (i - kF32B3)];
        else if (i < kF32B4) v = bf16r(P[kOffW4 + (i - kF32W4)]);
        else v = P[kOffB4];
        f32[i] = v;
    }
}

static spl_status prep(spl_mlp *m, cudaStream_t st)
{
    const int n = 2 * kHid * kRowWords;
    k_prep<<<(n + 255) / 256, 256, 0, st>>>(m->master, m->w23, m->f32, reinterpret_cast<TcMlpImage *>(m->tc_img));
    return cuda_check(cudaGetLastError(), "mlp prep launch");
}

// ---------------------------------------------------------------- batched evaluation
// FROM_WP: rows given as (omega, p) -> canonical features and the exact
// support mask of the basis at the origin; otherwise rows are features.
template <bool FROM_WP>
__global__ void __launch_bounds__(2 * kTcRows, 2) k_mlp_rows(MlpDev w, int degree, long long count,
                                                      const float *__restrict__ a, const float *__restrict__ b,
                                                      float *__restrict__ out)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcMlpSmem &S = *reinterpret_cast<TcMlpSmem *>(tc_smem);
    __shared__ float part[2 * kTcRows];
    tc_mlp_setup(w, S);
    unsigned phase = 0;
    const long long tiles = (count + kTcRows - 1) / kTcRows;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long r = tile * kTcRows + tc_rowid<2>();
        float x[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float mask = 0.0f;
        if (r < count) {
            mask = 1.0f;
            if (FROM_WP) {
                float wv[3], pv[3];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    wv[e] = a[3 * r + e];
                    pv[e] = b[3 * r + e];
                }
                const float inrm = rsqrtf(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
#pragma unroll
                for (int e = 0; e < 3; ++e) wv[e] *= inrm;
                canonical_features_f32(degree, wv, pv, x);
                // exact support: the line p + t w meets the open cube
                // [-W, W]^3 in a segment of positive length
                const float W = 0.5f * (degree + 1);
                float lo = -INFINITY, hi = INFINITY;
                bool in = true;
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if (wv[e] == 0.0f) {
                        in = in && (pv[e] >= -W && pv[e] < W) && (degree == 0 || pv[e] > -W);
                    } else {
                        const float iw = 1.0f / wv[e];
                        const float t1 = (-W - pv[e]) * iw, t2 = (W - pv[e]) * iw;
                        lo = fmaxf(lo, fminf(t1, t2));
                        hi = fminf(hi, fmaxf(t1, t2));
                    }
                }
                mask = (in && hi > lo) ? 1.0f : 0.0f;
            } else {
#pragma unroll
                for (int e = 0; e < 5; ++e) x[e] = a[5 * r + e];
            }
        }
        float o;
        const bool ok = tc_mlp_tile<2>(S, x, o, phase, part);
        // a tensor-core wait that gave up (not expected) leaves NaN in the
        // rows of the tile, sets the network's error flag and stops the CTA
        const bool bad = __syncthreads_or(!ok);
        if (r < count && tc_half<2>() == 0) out[r] = bad ? __int_as_float(0x7FC00000) : o * mask;
        if (bad) {
            if (threadIdx.x == 0) atomicOr(w.err, kErrTimeout);
            tc_mlp_teardown(S, phase, true);
            return;
        }
    }
    tc_mlp_teardown(S);
}

static unsigned eval_blocks(long long count)
{
    const long long tiles = (count + kTcRows - 1) / kTcRows;
    const long long cap = 4LL * sm_count();
    return (unsigned)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

// dynamic shared memory of the tcgen05 row kernels (set once per process)
template <bool FROM_WP> static spl_status rows_smem_attr()
{
    return smem_attr_once((const void *)k_mlp_rows<FROM_WP>, (int)sizeof(TcMlpSmem), "mlp rows smem attribute");
}

spl_status footprint_mlp(const spl_basis_desc *b, long long count, const float *w, const float *p, float *out,
                         cudaStream_t st)
{
    spl_status s = rows_smem_attr<true>();
    if (s != SPL_OK) return s;
    k_mlp_rows<true><<<eval_blocks(count), 2 * kTcRows, sizeof(TcMlpSmem), st>>>(mlp_dev(b->mlp), b->degree, count, w, p,
                                                                             out);
    return cuda_check(cudaGetLastError(), "mlp footprint launch");
}

// ---------------------------------------------------------------- training
__global__ void __launch_bounds__(2 * kTcRows, 2) k_train_forward(MlpDev w, int B, const float *__restrict__ X,
                                                               float *act, float *out, int max_batch)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    TcMlpSmem &S = *reinterpret_cast<TcMlpSmem *>(tc_smem);
    __shared__ float part[2 * kTcRows];
    tc_mlp_setup(w, S);
    unsigned phase = 0;
    const size_t L = (size_t)max_batch * 64;
    const int tiles = (B + kTcRows - 1) / kTcRows;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int r = tile * kTcRows + tc_rowid<2>();
        float x[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) x[e] = r < B ? X[5 * r + e] : 0.0f;
        const TcSave sv{act, act + L, act + 2 * L, act + 3 * L, act + 4 * L, act + 5 * L, r < B ? r : -1};
        float o;
        const bool ok = tc_mlp_tile<2, true>(S, x, o, phase, part, &sv);
        // a tensor-core wait that gave up (not expected) leaves NaN outputs,
        // so the loss and the gradient come out NaN, and sets the network's
        // error flag
        const bool bad = __syncthreads_or(!ok);
        if (r < B && tc_half<2>() == 0) out[r] = bad ? __int_as_float(0x7FC00000) : o;
        if (bad) {
            if (threadIdx.x == 0) atomicOr(w.err, kErrTimeout);
            tc_mlp_teardown(S, phase, true);
            return;
        }
    }
    tc_mlp_teardown(S);
}

__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// dL/dz of every layer for L = (1/B) sum (f(x_b) - y_b)^2.  Four threads
// per row (consecutive lanes), each owning 16 of the 64 units of a layer;
// a layer's gradient vector passes between them through shared memory
// (rows padded to 65 floats: the 8 rows of a warp hit distinct banks).
// Weights as used in the forward (BF16-rounded) come from the FP32 master
// rounded on the fly; roundings of activations pass straight through.
constexpr int kBwdThreads = 64;
constexpr int kBwdSplit = 4;                         // threads per row
constexpr int kBwdRows = kBwdThreads / kBwdSplit;    // rows per block
constexpr int kBwdUnits = kHid / kBwdSplit;          // units per thread

// gout[i] = silu'(z[i]) * sum_c W[c][i] gin[c] for this thread's units
// i = i0 .. i0 + 15; W as [c][i] (row c = output unit of the layer above)
__device__ __forceinline__ void back_layer(const float *__restrict__ W, const float *__restrict__ gin, int i0,
                                           const float *__restrict__ z, float *__restrict__ gout_g,
                                           float *__restrict__ gout_s)
{
    float acc[kBwdUnits];
#pragma unroll
    for (int q = 0; q < kBwdUnits; ++q) acc[q] = 0.0f;
#pragma unroll 8
    for (int c = 0; c < kHid; ++c) {
        const float g = gin[c];
        const float4 *w = reinterpret_cast<const float4 *>(W + c * kHid + i0);
#pragma unroll
        for (int q4 = 0; q4 < kBwdUnits / 4; ++q4) {
            const float4 v = w[q4];
            acc[4 * q4] = fmaf(v.x, g, acc[4 * q4]);
            acc[4 * q4 + 1] = fmaf(v.y, g, acc[4 * q4 + 1]);
            acc[4 * q4 + 2] = fmaf(v.z, g, acc[4 * q4 + 2]);
            acc[4 * q4 + 3] = fmaf(v.w, g, acc[4 * q4 + 3]);
        }
    }
#pragma unroll
    for (int q4 = 0; q4 < kBwdUnits / 4; ++q4) {
        const float4 zz = *reinterpret_cast<const float4 *>(z + i0 + 4 * q4);
        const float4 g = make_float4(acc[4 * q4] * silu_grad(zz.x), acc[4 * q4 + 1] * silu_grad(zz.y),
                                     acc[4 * q4 + 2] * silu_grad(zz.z), acc[4 * q4 + 3] * silu_grad(zz.w));
        *reinterpret_cast<float4 *>(gout_g + i0 + 4 * q4) = g;
        gout_s[i0 + 4 * q4] = g.x;
        gout_s[i0 + 4 * q4 + 1] = g.y;
        gout_s[i0 + 4 * q4 + 2] = g.z;
        gout_s[i0 + 4 * q4 + 3] = g.w;
    }
}

__global__ void __launch_bounds__(kBwdThreads) k_train_backward(const float *__restrict__ P, int B,
                                                                const float *__restrict__ Y,
                                                                const float *__restrict__ act,
                                                                const float *__restrict__ out, float *dz, float *dz4,
                                                                double *loss_part, int max_batch)
{
    // W2, W3 stored as [c][i] = W[c][i] (row c = output unit): reading
    // W[c][i0..i0+3] for fixed c is a float4
    __shared__ __align__(16) float W2[kHid * kHid];
    __shared__ __align__(16) float W3[kHid * kHid];
    __shared__ float W4[kHid];
    __shared__ float gbuf[2][kBwdRows][kHid + 1];
    __shared__ double red[kBwdThreads / 32];
    for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
        W2[i] = bf16r(P[kOffW2 + i]);
        W3[i] = bf16r(P[kOffW3 + i]);
    }
    if (threadIdx.x < kHid) W4[threadIdx.x] = bf16r(P[kOffW4 + threadIdx.x]);
    __syncthreads();
    const int lr = threadIdx.x / kBwdSplit, i0 = (threadIdx.x % kBwdSplit) * kBwdUnits;
    const int r = blockIdx.x * kBwdRows + lr;
    const size_t L = (size_t)max_batch * 64;
    double l2 = 0.0;
    const bool live = r < B;  // the four threads of a row agree
    if (live) {
        const float res = out[r] - Y[r];
        if (i0 == 0) {
            l2 = (double)res * res;
            dz4[r] = 2.0f * res / (float)B;
        }
        const float d4 = 2.0f * res / (float)B;
        const float *z3 = act + 4 * L + (size_t)r * 64;
#pragma unroll
        for (int c = i0; c < i0 + kBwdUnits; c += 4) {
            const float4 zz = *reinterpret_cast<const float4 *>(z3 + c);
            const float4 g = make_float4(W4[c] * d4 * silu_grad(zz.x), W4[c + 1] * d4 * silu_grad(zz.y),
                                         W4[c + 2] * d4 * silu_grad(zz.z), W4[c + 3] * d4 * silu_grad(zz.w));
            *reinterpret_cast<float4 *>(dz + 2 * L + (size_t)r * 64 + c) = g;
            gbuf[0][lr][c] = g.x;
            gbuf[0][lr][c + 1] = g.y;
            gbuf[0][lr][c + 2] = g.z;
            gbuf[0][lr][c + 3] = g.w;
        }
    }
    __syncwarp();
    if (live) back_layer(W3, gbuf[0][lr], i0, act + 2 * L + (size_t)r * 64, dz + L + (size_t)r * 64, gbuf[1][lr]);
    __syncwarp();
    if (live) back_layer(W2, gbuf[1][lr], i0, act + (size_t)r * 64, dz + (size_t)r * 64, gbuf[0][lr]);
    // per-block loss partial (fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_down_sync(0xffffffffu, l2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBwdThreads / 32; ++w) t += red[w];
        loss_part[blockIdx.x] = t;
    }
}

// Weight gradients of one batch chunk: block (chunk, layer).  Rows are
// staged through shared memory 32 at a time; for the 64x64 layers each
// thread owns one output unit o and 16 consecutive inputs, and sums the
// chunk's rows in order (deterministic).
constexpr int kStageRows = 32;

__global__ void __launch_bounds__(kWgThreads) k_train_wgrad(int B, const float *__restrict__ X,
                                                            const float *__restrict__ act,
                                                            const float *__restrict__ dz,
                                                            const float *__restrict__ dz4, float *part, int max_batch)
{
    __shared__ __align__(16) float Gs[kStageRows][kHid];
    __shared__ __align__(16) float Hs[kStageRows][kHid];
    const int chunk = blockIdx.x, layer = blockIdx.y;
    const size_t L = (size_t)max_batch * 64;
    const int r0 = chunk * kChunkRows, r1 = min(B, r0 + kChunkRows);
    float *dst = part + (size_t)chunk * (kParams + 1);
    int nin, nout, offW, offB, hstride, gstride;
    const float *H, *G;
    if (layer == 0) { nin = kIn; nout = kHid; H = X; hstride = kIn; G = dz; gstride = 64; offW = kOffW1; offB = kOffB1; }
    else if (layer == 1) { nin = kHid; nout = kHid; H = act + L; hstride = 64; G = dz + L; gstride = 64; offW = kOffW2; offB = kOffB2; }
    else if (layer == 2) { nin = kHid; nout = kHid; H = act + 3 * L; hstride = 64; G = dz + 2 * L; gstride = 64; offW = kOffW3; offB = kOffB3; }
    else { nin = kHid; nout = 1; H = act + 5 * L; hstride = 64; G = dz4; gstride = 1; offW = kOffW4; offB = kOffB4; }
    // thread -> (o, 16 inputs starting at i0); the thread with i0 = 0 also
    // sums the bias gradient of o
    const int nslots = nout * ((nin + 15) / 16);
    const int slot = threadIdx.x;
    const bool has_w = slot < nslots;
    const int o = has_w ? slot / ((nin + 15) / 16) : 0;
    const int i0 = has_w ? (slot % ((nin + 15) / 16)) * 16 : 0;
    const bool has_b = has_w && i0 == 0;
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    float accb = 0.0f;
    for (int rs = r0; rs < r1; rs += kStageRows) {
        const int nr = min(kStageRows, r1 - rs);
        __syncthreads();
        for (int e = threadIdx.x; e < kStageRows * kHid; e += blockDim.x) {
            const int rr = e / kHid, cc = e % kHid;
            Gs[rr][cc] = (rr < nr && cc < nout) ? G[(size_t)(rs + rr) * gstride + cc] : 0.0f;
            Hs[rr][cc] = (rr < nr && cc < nin) ? H[(size_t)(rs + rr) * hstride + cc] : 0.0f;
        }
        __syncthreads();
        if (has_w) {
            for (int rr = 0; rr < nr; ++rr) {
                const float gv = Gs[rr][o];
                accb += gv;
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = fmaf(gv, Hs[rr][i0 + q], acc[q]);
            }
        }
    }
    if (has_w) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (i0 + q < nin) dst[offW + o * nin + i0 + q] = acc[q];
        if (has_b) dst[offB + o] = accb;
    }
}

// Gradient and loss from the partials in a fixed order: block b owns 32
// parameters; warp w sums chunks w, w + 8, ... in order, then warp 0 adds
// the 8 sums in order.  Block 0 also sums the loss partials (thread t:
// partials t, t + 256, ...; then 8 per lane and a fixed shuffle tree).
constexpr int kRedThreads = 256;
__global__ void __launch_bounds__(kRedThreads) k_train_reduce(const float *__restrict__ part, int chunks,
                                                              const double *__restrict__ loss_part, int nloss, int B,
                                                              float *grad, float *loss_out)
{
    __shared__ float ps[kRedThreads / 32][32];
    __shared__ double ls[kRedThreads];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float acc = 0.0f;
    if (i < kParams)
        for (int c = w; c < chunks; c += kRedThreads / 32) acc += part[(size_t)c * (kParams + 1) + i];
    ps[w][lane] = acc;
    const bool do_loss = blockIdx.x == 0 && loss_out != nullptr;
    if (do_loss) {
        double l = 0.0;
        for (int k = threadIdx.x; k < nloss; k += kRedThreads) l += loss_part[k];
        ls[threadIdx.x] = l;
    }
    __syncthreads();
    if (w == 0) {
        if (i < kParams) {
            float t = 0.0f;
#pragma unroll
            for (int g = 0; g < kRedThreads / 32; ++g) t += ps[g][lane];
            grad[i] = t;
        }
        if (do_loss) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < kRedThreads / 32; ++k) t += ls[lane * (kRedThreads / 32) + k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) loss_out[0] = (float)(t / (double)B);
        }
    }
}

__global__ void k_adam(float *P, float *m, float *v, const float *__restrict__ g, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

static spl_status grad_impl(spl_mlp *m, int B, const float *X, const float *Y, float *grad, float *loss,
                            cudaStream_t st)
{
    const MlpDev w = mlp_dev(m);
    {
        spl_status s = smem_attr_once((const void *)k_train_forward, (int)sizeof(TcMlpSmem),
                                      "train forward smem attribute");
        if (s != SPL_OK) return s;
    }
    k_train_forward<<<eval_blocks(B), 2 * kTcRows, sizeof(TcMlpSmem), st>>>(w, B, X, m->act, m->out, m->max_batch);
    const int bblocks = (B + kBwdRows - 1) / kBwdRows;
    k_train_backward<<<bblocks, kBwdThreads, 0, st>>>(m->master, B, Y, m->act, m->out, m->dz, m->dz4, m->loss_part,
                                                      m->max_batch);
    const int chunks = (B + kChunkRows - 1) / kChunkRows;
    k_train_wgrad<<<dim3(chunks, 4), kWgThreads, 0, st>>>(B, X, m->act, m->dz, m->dz4, m->part, m->max_batch);
    k_train_reduce<<<(kParams + 31) / 32, kRedThreads, 0, st>>>(m->part, chunks, m->loss_part, bblocks, B, grad, loss);
    return cuda_check(cudaGetLastError(), "mlp gradient launch");
}

// SplitMix64 (Steele, Lea and Flood 2014): seeded initial parameters.
static uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

}  // namespace spl

using namespace spl;

extern "C" int spl_mlp_degree(const spl_mlp *m) { return m ? m->degree : -1; }

extern "C" spl_status spl_mlp_create(int degree, int max_batch, unsigned long long seed, spl_mlp **out)
{
    clear_error();
    if (!out) return fail(SPL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (degree < 0 || degree > 3) return fail(SPL_ERR_ARG, "degree %d not in 0..3", degree);
    if (max_batch < 16 || max_batch > (1 << 22)) return fail(SPL_ERR_ARG, "max_batch %d not in 16..2^22", max_batch);
    spl_mlp *m = (spl_mlp *)calloc(1, sizeof(spl_mlp));
    if (!m) return fail(SPL_ERR_OOM, "host allocation failed");
    m->degree = degree;
    m->max_batch = max_batch;
    m->seed = seed;
    cudaGetDevice(&m->device);
    const int chunks = (max_batch + kChunkRows - 1) / kChunkRows;
    const int nloss = (max_batch + kBwdRows - 1) / kBwdRows;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_master = take(kParams * 4), o_m = take(kParams * 4), o_v = take(kParams * 4),
                 o_grad = take(kParams * 4), o_w23 = take(2 * kHid * kRowWords * 4), o_f32 = take(kF32Size * 4),
                 o_img = take(sizeof(TcMlpImage)),
                 o_act = take((size_t)6 * max_batch * 64 * 4), o_out = take((size_t)max_batch * 4),
                 o_dz = take((size_t)3 * max_batch * 64 * 4), o_dz4 = take((size_t)max_batch * 4),
                 o_part = take((size_t)chunks * (kParams + 1) * 4), o_loss = take((size_t)nloss * 8),
                 o_err = take(sizeof(int));
    void *blk = nullptr;
    cudaError_t ce = cudaMalloc(&blk, off);
    if (ce != cudaSuccess) {
        free(m);
        cudaGetLastError();
        return fail(SPL_ERR_OOM, "cudaMalloc(%zu) failed: %s", off, cudaGetErrorString(ce));
    }
    char *base = (char *)blk;
    m->block = blk;
    m->master = (float *)(base + o_master);
    m->adam_m = (float *)(base + o_m);
    m->adam_v = (float *)(base + o_v);
    m->grad = (float *)(base + o_grad);
    m->w23 = (uint32_t *)(base + o_w23);
    m->f32 = (float *)(base + o_f32);
    m->tc_img = base + o_img;
    m->act = (float *)(base + o_act);
    m->out = (float *)(base + o_out);
    m->dz = (float *)(base + o_dz);
    m->dz4 = (float *)(base + o_dz4);
    m->part = (float *)(base + o_part);
    m->loss_part = (double *)(base + o_loss);
    m->err = (int *)(base + o_err);
    if (cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(blk);
        free(m);
        return fail(SPL_ERR_CUDA, "error flag clear failed");
    }
    // seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) for weights and biases
    float *h = (float *)malloc(kParams * sizeof(float));
    if (!h) { cudaFree(blk); free(m); return fail(SPL_ERR_OOM, "host allocation failed"); }
    uint64_t st = seed;
    const int fan_in[4] = {kIn, kHid, kHid, kHid};
    const int offs[5] = {0, kOffW2, kOffW3, kOffW4, kParams};
    for (int layer = 0; layer < 4; ++layer) {
        const float bound = 1.0f / sqrtf((float)fan_in[layer]);
        for (int i = offs[layer]; i < offs[layer + 1]; ++i) {
            const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
            h[i] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    spl_status s = spl_mlp_set_params(m, h);
    free(h);
    if (s != SPL_OK) {
        cudaFree(blk);
        free(m);
        return s;
    }
    *out = m;
    return SPL_OK;
}

extern "C" void spl_mlp_destroy(spl_mlp *m)
{
    if (!m) return;
    if (m->block) cudaFree(m->block);
    free(m);
}

extern "C" spl_status spl_mlp_set_params(spl_mlp *m, const float *host_params)
{
    clear_error();
    if (!m || !host_params) return fail(SPL_ERR_ARG, "NULL argument");
    for (int i = 0; i < kParams; ++i)
        if (!isfinite(host_params[i])) return fail(SPL_ERR_NONFINITE, "parameter %d is not finite", i);
    spl_status s = cuda_check(cudaMemcpy(m->master, host_params, kParams * 4, cudaMemcpyHostToDevice), "params upload");
    if (s != SPL_OK) return s;
    s = cuda_check(cudaMemset(m->adam_m, 0, kParams * 4), "adam reset");
    if (s != SPL_OK) return s;
    s = cuda_check(cudaMemset(m->adam_v, 0, kParams * 4), "adam reset");
    if (s != SPL_OK) return s;
    m->step = 0;
    s = prep(m, 0);
    if (s != SPL_OK) return s;
    return cuda_check(cudaDeviceSynchronize(), "params prep");
}

extern "C" spl_status spl_mlp_status(const spl_mlp *m, void *stream)
{
    clear_error();
    if (!m) return fail(SPL_ERR_ARG, "mlp is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    spl_status s = cuda_check(cudaMemcpyAsync(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost, st), "status read");
    if (s == SPL_OK) s = cuda_check(cudaStreamSynchronize(st), "status sync");
    if (s != SPL_OK) return s;
    if (flag) {
        s = cuda_check(cudaMemsetAsync(m->err, 0, sizeof(int), st), "status clear");
        if (s == SPL_OK) s = cuda_check(cudaStreamSynchronize(st), "status sync");
        if (s != SPL_OK) return s;
        return fail(SPL_ERR_TIMEOUT, "a bounded tensor-core wait gave up (flag 0x%x)", flag);
    }
    return SPL_OK;
}

// ---------------------------------------------------------------- checkpoint
namespace {
const char kCkptMagic[8] = {'S', 'P', 'L', 'M', 'L', 'P', '2', '\0'};
constexpr int kCkptVersion = 2;
constexpr int kCkptHeader = 8;  // int32 fields after the magic

void put_le32(unsigned char *b, uint32_t v)
{
    for (int i = 0; i < 4; ++i) b[i] = (unsigned char)(v >> (8 * i));
}
uint32_t get_le32(const unsigned char *b)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)b[i] << (8 * i);
    return v;
}
}  // namespace

extern "C" spl_status spl_mlp_save(const spl_mlp *m, const char *path)
{
    clear_error();
    if (!m || !path) return fail(SPL_ERR_ARG, "NULL argument");
    const size_t nbytes = 8 + 4 * kCkptHeader + 8 + 3 * (size_t)kParams * 4;
    unsigned char *buf = (unsigned char *)malloc(nbytes);
    if (!buf) return fail(SPL_ERR_OOM, "host allocation failed");
    memcpy(buf, kCkptMagic, 8);
    const int32_t head[kCkptHeader] = {kCkptVersion, m->degree, kParams, kIn, kHid, 3, 0, m->step};
    for (int i = 0; i < kCkptHeader; ++i) put_le32(buf + 8 + 4 * i, (uint32_t)head[i]);
    unsigned char *p = buf + 8 + 4 * kCkptHeader;
    put_le32(p, (uint32_t)(m->seed & 0xffffffffu));
    put_le32(p + 4, (uint32_t)(m->seed >> 32));
    p += 8;
    float *tmp = (float *)malloc((size_t)kParams * 4);
    if (!tmp) {
        free(buf);
        return fail(SPL_ERR_OOM, "host allocation failed");
    }
    const float *src[3] = {m->master, m->adam_m, m->adam_v};
    spl_status s = cuda_check(cudaDeviceSynchronize(), "checkpoint sync");
    for (int a = 0; a < 3 && s == SPL_OK; ++a) {
        s = cuda_check(cudaMemcpy(tmp, src[a], (size_t)kParams * 4, cudaMemcpyDeviceToHost), "checkpoint download");
        for (int i = 0; i < kParams && s == SPL_OK; ++i) {
            uint32_t bits;
            memcpy(&bits, tmp + i, 4);
            put_le32(p + 4 * ((size_t)a * kParams + i), bits);
        }
    }
    free(tmp);
    if (s == SPL_OK) {
        FILE *f = fopen(path, "wb");
        if (!f) s = fail(SPL_ERR_ARG, "cannot open %s for writing", path);
        else {
            const size_t w = fwrite(buf, 1, nbytes, f);
            const int c = fclose(f);
            if (w != nbytes || c != 0) s = fail(SPL_ERR_ARG, "write to %s failed", path);
        }
    }
    free(buf);
    return s;
}

extern "C" spl_status spl_mlp_load(spl_mlp *m, const char *path)
{
    clear_error();
    if (!m || !path) return fail(SPL_ERR_ARG, "NULL argument");
    const size_t nbytes = 8 + 4 * kCkptHeader + 8 + 3 * (size_t)kParams * 4;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(SPL_ERR_ARG, "cannot open %s", path);
    unsigned char *buf = (unsigned char *)malloc(nbytes + 1);
    if (!buf) {
        fclose(f);
        return fail(SPL_ERR_OOM, "host allocation failed");
    }
    const size_t got = fread(buf, 1, nbytes + 1, f);
    fclose(f);
    spl_status s = SPL_OK;
    int32_t head[kCkptHeader];
    if (got != nbytes) s = fail(SPL_ERR_ARG, "%s: %zu bytes, expected %zu", path, got, nbytes);
    else if (memcmp(buf, kCkptMagic, 8) != 0) s = fail(SPL_ERR_ARG, "%s is not an f_theta checkpoint", path);
    if (s == SPL_OK) {
        for (int i = 0; i < kCkptHeader; ++i) head[i] = (int32_t)get_le32(buf + 8 + 4 * i);
        if (head[0] != kCkptVersion || head[2] != kParams || head[3] != kIn || head[4] != kHid || head[5] != 3 ||
            head[6] != 0)
            s = fail(SPL_ERR_ARG, "%s: unsupported version or network shape", path);
        else if (head[1] != m->degree)
            s = fail(SPL_ERR_ARG, "%s holds a network for degree %d, not %d", path, head[1], m->degree);
        else if (head[7] < 0)
            s = fail(SPL_ERR_ARG, "%s: negative step count", path);
    }
    float *vals = nullptr;
    if (s == SPL_OK) {
        vals = (float *)malloc(3 * (size_t)kParams * 4);
        if (!vals) s = fail(SPL_ERR_OOM, "host allocation failed");
    }
    if (s == SPL_OK) {
        const unsigned char *p = buf + 8 + 4 * kCkptHeader + 8;
        for (size_t i = 0; i < 3 * (size_t)kParams; ++i) {
            const uint32_t bits = get_le32(p + 4 * i);
            memcpy(vals + i, &bits, 4);
            if (!isfinite(vals[i])) {
                s = fail(SPL_ERR_NONFINITE, "%s: value %zu is not finite", path, i);
                break;
            }
        }
    }
    if (s == SPL_OK) {
        const unsigned char *p = buf + 8 + 4 * kCkptHeader;
        float *dst[3] = {m->master, m->adam_m, m->adam_v};
        s = cuda_check(cudaDeviceSynchronize(), "checkpoint sync");
        for (int a = 0; a < 3 && s == SPL_OK; ++a)
            s = cuda_check(cudaMemcpy(dst[a], vals + (size_t)a * kParams, (size_t)kParams * 4, cudaMemcpyHostToDevice),
                           "checkpoint upload");
        if (s == SPL_OK) {
            m->step = head[7];
            m->seed = (unsigned long long)get_le32(p) | ((unsigned long long)get_le32(p + 4) << 32);
            s = prep(m, 0);
        }
        if (s == SPL_OK) s = cuda_check(cudaDeviceSynchronize(), "checkpoint prep");
    }
    free(vals);
    free(buf);
    return s;
}

extern "C" spl_status spl_mlp_get_params(const spl_mlp *m, float *host_params)
{
    clear_error();
    if (!m || !host_params) return fail(SPL_ERR_ARG, "NULL argument");
    return cuda_check(cudaMemcpy(host_params, m->master, kParams * 4, cudaMemcpyDeviceToHost), "params download");
}

extern "C" spl_status spl_mlp_eval(const spl_mlp *m, long long count, const float *feat_dev, float *out_dev,
                                   void *stream)
{
    clear_error();
    if (!m) return fail(SPL_ERR_ARG, "mlp is NULL");
    if (count < 0) return fail(SPL_ERR_ARG, "bad count");
    if (count == 0) return SPL_OK;
    if (!feat_dev || !out_dev) return fail(SPL_ERR_ARG, "NULL array");
    spl_status s = rows_smem_attr<false>();
    if (s != SPL_OK) return s;
    k_mlp_rows<false><<<eval_blocks(count), 2 * kTcRows, sizeof(TcMlpSmem), (cudaStream_t)stream>>>(
        mlp_dev(m), m->degree, count, feat_dev, nullptr, out_dev);
    return cuda_check(cudaGetLastError(), "mlp eval launch");
}

extern "C" spl_status spl_mlp_grad(spl_mlp *m, int batch, const float *feat_dev, const float *target_dev,
                                   float *grad_dev, float *loss_dev, void *stream)
{
    clear_error();
    if (!m || !feat_dev || !target_dev || !grad_dev) return fail(SPL_ERR_ARG, "NULL argument");
    if (batch < 1 || batch > m->max_batch) return fail(SPL_ERR_ARG, "batch %d not in 1..%d", batch, m->max_batch);
    return grad_impl(m, batch, feat_dev, target_dev, grad_dev, loss_dev, (cudaStream_t)stream);
}

extern "C" spl_status spl_mlp_train_step(spl_mlp *m, int batch, const float *feat_dev, const float *target_dev,
                                         float lr, float *loss_dev, void *stream)
{
    clear_error();
    if (!m || !feat_dev || !target_dev) return fail(SPL_ERR_ARG, "NULL argument");
    if (batch < 1 || batch > m->max_batch) return fail(SPL_ERR_ARG, "batch %d not in 1..%d", batch, m->max_batch);
    if (!(lr >= 0.0f) || !isfinite(lr)) return fail(SPL_ERR_ARG, "bad learning rate");
    cudaStream_t st = (cudaStream_t)stream;
    spl_status s = grad_impl(m, batch, feat_dev, target_dev, m->grad, loss_dev, st);
    if (s != SPL_OK) return s;
    m->step += 1;
    const float c1 = 1.0f - powf(0.9f, (float)m->step), c2 = 1.0f - powf(0.999f, (float)m->step);
    k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(m->master, m->adam_m, m->adam_v, m->grad, lr, c1, c2);
    s = cuda_check(cudaGetLastError(), "adam launch");
    if (s != SPL_OK) return s;
    return prep(m, st);
}
