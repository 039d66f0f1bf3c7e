// blas.cu -- FP64 reductions and vector updates of least-squares
// reconstruction (Eq. 5, solved by CGLS on the normal equations).
//
// spl_dot_f64 is deterministic: a fixed grid of blocks (independent of n)
// accumulates grid-strided products in FP64, each block writes one partial
// to the caller's workspace, and a single block adds the partials in index
// order.  The CG updates read their FP64 scalars from device memory, so an
// iteration needs no host synchronisation.
#include <mutex>

#include "spl_host.h"

namespace spl {

constexpr int kDotBlocks = 1024;
constexpr int kDotThreads = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__global__ void __launch_bounds__(kDotThreads) k_dot_partial(long long n, const float *__restrict__ a,
                                                             const float *__restrict__ b, double *__restrict__ part)
{
    __shared__ double sh[kDotThreads / 32];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // 4 independent FP64 accumulators per thread for memory-level parallelism
    double a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (; i + 3 * stride < n; i += 4 * stride) {
        acc = fma((double)__ldg(a + i), (double)__ldg(b + i), acc);
        a1 = fma((double)__ldg(a + i + stride), (double)__ldg(b + i + stride), a1);
        a2 = fma((double)__ldg(a + i + 2 * stride), (double)__ldg(b + i + 2 * stride), a2);
        a3 = fma((double)__ldg(a + i + 3 * stride), (double)__ldg(b + i + 3 * stride), a3);
    }
    for (; i < n; i += stride) acc = fma((double)__ldg(a + i), (double)__ldg(b + i), acc);
    acc = (acc + a1) + (a2 + a3);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kDotThreads) k_dot_final(const double *__restrict__ part, int np, double *out)
{
    __shared__ double sh[kDotThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = acc;
}

// x += alpha p ; r -= alpha q  (alpha = num / den, 0 if den == 0)
__global__ void k_cg_step_x(long long nx, float *__restrict__ x, const float *__restrict__ p, long long nr,
                            float *__restrict__ r, const float *__restrict__ q, const double *num, const double *den)
{
    const double dd = *den;
    const float alpha = dd != 0.0 ? (float)(*num / dd) : 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += stride)
        x[i] = fmaf(alpha, p[i], x[i]);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride)
        r[i] = fmaf(-alpha, q[i], r[i]);
}

// p = s + beta p  (beta = num / den, 0 if den == 0)
__global__ void k_cg_step_p(long long n, float *__restrict__ p, const float *__restrict__ s, const double *num,
                            const double *den)
{
    const double dd = *den;
    const float beta = dd != 0.0 ? (float)(*num / dd) : 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = fmaf(beta, p[i], s[i]);
}

static int stream_blocks(long long n)
{
    const long long b = (n + 255) / 256, cap = 8LL * sm_count();
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// FP32 throughput probe: kProbeChains independent FMA chains per thread,
// x <- x a + b (contracting to b / (1 - a): no overflow, no subnormals), as
// scalar FMAs or as packed FP32x2 FMAs (__ffma2_rn, two per instruction).
constexpr int kProbeChains = 16;
constexpr int kProbeThreads = 256;
__global__ void __launch_bounds__(kProbeThreads) k_fp32_probe(int iters, int packed, float *out)
{
    const float a = 0.9999f, b = 1e-4f;
    const float x0 = 0.5f + 1e-6f * (float)(threadIdx.x + blockIdx.x);
    float sum = 0.0f;
    if (packed) {
        float2 x[kProbeChains / 2];
#pragma unroll
        for (int i = 0; i < kProbeChains / 2; ++i) x[i] = make_float2(x0 + 0.01f * i, x0 - 0.01f * i);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 1
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < kProbeChains / 2; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
        }
#pragma unroll
        for (int i = 0; i < kProbeChains / 2; ++i) sum += x[i].x + x[i].y;
    } else {
        float x[kProbeChains];
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) x[i] = x0 + 0.01f * i;
#pragma unroll 1
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < kProbeChains; ++i) x[i] = fmaf(x[i], a, b);
        }
#pragma unroll
        for (int i = 0; i < kProbeChains; ++i) sum += x[i];
    }
    if (sum == -1.0f) out[0] = sum;  // never true; keeps the chains live
}

}  // namespace spl

using namespace spl;

extern "C" long long spl_dot_f64_workspace_bytes(void) { return (long long)kDotBlocks * sizeof(double); }

extern "C" spl_status spl_fp32_probe(int packed, int blocks_per_sm, int iters, float *out_dev, double *flop,
                                     void *stream)
{
    clear_error();
    if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !out_dev || !flop)
        return fail(SPL_ERR_ARG, "bad argument");
    const int blocks = blocks_per_sm * sm_count();
    *flop = 2.0 * 4.0 * kProbeChains * (double)iters * blocks * kProbeThreads;
    k_fp32_probe<<<blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(iters, packed ? 1 : 0, out_dev);
    return cuda_check(cudaGetLastError(), "probe launch");
}

extern "C" int spl_sm_count(void) { return sm_count(); }

extern "C" spl_status spl_dot_f64(long long n, const float *a_dev, const float *b_dev, double *out_dev, void *work_dev,
                                  long long work_bytes, void *stream)
{
    clear_error();
    if (n < 0) return fail(SPL_ERR_ARG, "negative length");
    if (!out_dev || !work_dev || (n > 0 && (!a_dev || !b_dev))) return fail(SPL_ERR_ARG, "NULL pointer");
    if (work_bytes < spl_dot_f64_workspace_bytes())
        return fail(SPL_ERR_ARG, "workspace of %lld bytes < %lld", work_bytes, spl_dot_f64_workspace_bytes());
    cudaStream_t st = (cudaStream_t)stream;
    double *part = (double *)work_dev;
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(n, a_dev, b_dev, part);
    k_dot_final<<<1, kDotThreads, 0, st>>>(part, kDotBlocks, out_dev);
    return cuda_check(cudaGetLastError(), "dot launch");
}

extern "C" spl_status spl_cg_step_x(long long nx, float *x_dev, const float *p_dev, long long nr, float *r_dev,
                                    const float *q_dev, const double *num_dev, const double *den_dev, void *stream)
{
    clear_error();
    if (nx < 0 || nr < 0 || !x_dev || !p_dev || !r_dev || !q_dev || !num_dev || !den_dev)
        return fail(SPL_ERR_ARG, "bad argument");
    const long long m = nx > nr ? nx : nr;
    k_cg_step_x<<<stream_blocks(m), 256, 0, (cudaStream_t)stream>>>(nx, x_dev, p_dev, nr, r_dev, q_dev, num_dev, den_dev);
    return cuda_check(cudaGetLastError(), "cg step launch");
}

extern "C" spl_status spl_cg_step_p(long long n, float *p_dev, const float *s_dev, const double *num_dev,
                                    const double *den_dev, void *stream)
{
    clear_error();
    if (n < 0 || !p_dev || !s_dev || !num_dev || !den_dev) return fail(SPL_ERR_ARG, "bad argument");
    k_cg_step_p<<<stream_blocks(n), 256, 0, (cudaStream_t)stream>>>(n, p_dev, s_dev, num_dev, den_dev);
    return cuda_check(cudaGetLastError(), "cg step launch");
}

// ---------------------------------------------------------------------------
// Allocation-free inner product.  Some callers cannot let a library allocate
// device memory: host frameworks that own every byte of device memory
// through their own pool and forbid third-party allocations, programs with a
// device-memory budget fixed at start-up, and latency-critical loops that
// cannot afford the implicit device synchronisation of cudaMalloc.  For them
// spl_dot_f64_noalloc runs the same two kernels as spl_dot_f64 with the
// partial sums in a fixed file-scope device array instead of a caller
// workspace.
// ---------------------------------------------------------------------------
namespace {

// kDotBlocks FP64 partials (8 KB); every GPU that loads the library holds
// this array until the process exits.  Each block of k_dot_partial writes its
// own entry, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_dot_noalloc_scratch[spl::kDotBlocks];

constexpr int kMaxDevices = 64;
static double *g_dot_noalloc_ptr[kMaxDevices];
static std::mutex g_dot_noalloc_mutex;

// Device address of the scratch array on the current device.  The first call
// on a device looks it up (cudaGetSymbolAddress with that device current) and
// caches it; later calls reuse the cached address.
spl_status noalloc_scratch(double **out)
{
    int dev = 0;
    spl_status s = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != SPL_OK) return s;
    if (dev < 0 || dev >= kMaxDevices) return fail(SPL_ERR_UNSUPPORTED, "device index %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_dot_noalloc_mutex);
    if (!g_dot_noalloc_ptr[dev]) {
        double *ptr = nullptr;
        s = cuda_check(cudaGetSymbolAddress((void **)&ptr, g_dot_noalloc_scratch), "cudaGetSymbolAddress");
        if (s != SPL_OK) return s;
        g_dot_noalloc_ptr[dev] = ptr;
    }
    *out = g_dot_noalloc_ptr[dev];
    return SPL_OK;
}

}  // namespace

extern "C" spl_status spl_dot_f64_noalloc(long long n, const float *a_dev, const float *b_dev, double *out_dev,
                                          void *stream)
{
    clear_error();
    if (n < 0) return fail(SPL_ERR_ARG, "negative length");
    if (n > SPL_DOT_NOALLOC_MAX_N)
        return fail(SPL_ERR_ARG, "length %lld exceeds the allocation-free maximum of %lld elements", n,
                    (long long)SPL_DOT_NOALLOC_MAX_N);
    if (!out_dev || (n > 0 && (!a_dev || !b_dev))) return fail(SPL_ERR_ARG, "NULL pointer");
    double *part = nullptr;
    spl_status s = noalloc_scratch(&part);
    if (s != SPL_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, st>>>(n, a_dev, b_dev, part);
    k_dot_final<<<1, kDotThreads, 0, st>>>(part, kDotBlocks, out_dev);
    return cuda_check(cudaGetLastError(), "dot launch");
}
