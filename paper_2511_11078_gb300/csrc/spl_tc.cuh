// spl_tc.cuh -- the learned footprint f_theta (Sec. 2.2) on the 5th-generation
// tensor cores: tcgen05.mma with operands in shared memory and the FP32
// accumulator in tensor memory (TMEM).
//
// A CTA evaluates tiles of 128 rows, with one thread per row (128 threads)
// or two (256 threads, each taking half of the row's 64 columns).  Each
// layer is one M=128 x N=64 product: the threads write their parts of the A
// operand (BF16) to shared memory, one thread issues the MMAs, the tensor
// core accumulates the 128 x 64 FP32 result in 64 TMEM columns, and every
// thread reads its part back with tcgen05.ld (TMEM lane = row), applies
// SiLU and writes the next layer's A operand.  The MMAs take no issue slots
// of the other threads and no registers: what is left to the threads is
// SiLU, the BF16 packing and the 64 -> 1 output layer.
//
// Precision contract (the one the oracle emulates): layers 2 and 3 multiply
// BF16 weights with the BF16-rounded activations, accumulating in FP32;
// layer 1 and the biases keep FP32 accuracy through three-part BF16 splits
// x = hi + mid + lo (hi and mid truncate the mantissa to 8 bits, the
// differences being exact in FP32; lo rounds the remainder to nearest, so
// what is dropped is below 2^-23 |x|): layer 1 multiplies
// [hi(x), mid(x), lo(x), 0] (16 columns) with [W1; W1; W1; 0], and each
// bias enters through one more K=16 step whose A rows are (1, 1, 1, 0 ...)
// and whose B rows are (hi(b), mid(b), lo(b), 0 ...).  The output layer is
// FP32 on the CUDA cores.
//
// Operand layout: the canonical K-major layout without swizzling.  An
// operand of R rows and K columns (BF16) is made of 8-row x 16-byte core
// matrices; core matrix (row group i, column group j) sits at byte
// j * (R / 8) * 128 + i * 128, row r of it at + 16 r.  The shared-memory
// descriptor takes the distance between core matrices along K (leading
// byte offset, (R / 8) * 128) and along the rows (stride byte offset, 128).
#pragma once

#include <stddef.h>

#include "spl_mlp.cuh"

namespace spl {
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// Shared-memory matrix descriptor (tcgen05 format): start address, leading
// and stride byte offsets (all in 16-byte units), descriptor version 1 at
// bit 46, base offset 0, no swizzling.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) = A * B (+ D when acc), A and B from shared memory
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// arrive on the mbarrier once every MMA this thread issued so far is complete
__device__ __forceinline__ void commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

// Wait for the phase with the given parity to complete; gives up (false)
// after a bounded number of polls.
constexpr unsigned kWaitPolls = 1u << 20;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = saddr(bar);
    for (unsigned it = 0; it < kWaitPolls; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the
// tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// warp-wide: allocate ncols TMEM columns, base address written to *dst
__device__ __forceinline__ void alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (lane = thread)
// into v[O .. O + 31]
template <int O, int L>
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[L])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[O + i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace tc

constexpr int kTcRows = 128;  // rows of a tile (threads of a CTA: 128 or 256)
constexpr int kTcCols = 64;   // TMEM columns of the accumulator (N = 64, FP32)
// TMEM allocation never waits: every CTA that allocates holds at least
// sizeof(TcMlpSmem) (49 KB) of shared memory, so at most 4 of them are
// resident on an SM (228 KB), and 4 x 64 columns stay below the SM's 512.

// The network in the tile's operand layout (built once per parameter
// update in global memory, copied into every CTA's shared memory).
struct __align__(16) TcMlpImage {
    uint8_t w2[64 * 64 * 2];        // B of layer 2: 64 (N) x 64 (K)
    uint8_t w3[64 * 64 * 2];
    uint8_t w1[64 * 16 * 2];        // B of layer 1: 64 x 16, [W1; W1; W1; 0]
    uint8_t bias[3][64 * 16 * 2];   // B of the bias steps of layers 1-3
    uint8_t one[kTcRows * 16 * 2];  // A of the bias steps: rows (1, 1, 1, 0 ...)
    float w4[64];
    float b4;
    float pad[3];
};

// Shared memory of a CTA: the network image and the operands of one tile.
struct __align__(1024) TcMlpSmem {
    TcMlpImage img;
    uint8_t a2[kTcRows * 64 * 2];  // A of layers 2 and 3: 128 x 64
    uint8_t a1[kTcRows * 16 * 2];  // A of layer 1: 128 x 16
    uint32_t tmem;
    uint64_t mbar;
};

static_assert(sizeof(TcMlpImage) % 16 == 0, "the image is copied in 16-byte units");
static_assert(offsetof(TcMlpSmem, a2) % 16 == 0 && offsetof(TcMlpSmem, a1) % 16 == 0,
              "operands start on 16-byte boundaries (shared-memory descriptors)");
static_assert(5 * (sizeof(TcMlpSmem) + 1024) > 228 * 1024, "at most 4 allocating CTAs per SM");

// byte offset of element (row, k) in an operand of R rows (K-major, no swizzle)
__host__ __device__ constexpr uint32_t kmaj_off(int R, int row, int k)
{
    return (uint32_t)((k >> 3) * (R / 8) * 128 + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint16_t bf16_bits_rn(float x)
{
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t *>(&h);
}
// three-part split of an FP32 value (hi, mid truncated, lo rounded)
__device__ __forceinline__ void split3(float x, uint16_t &hi, uint16_t &mid, uint16_t &lo)
{
    const uint32_t bx = __float_as_uint(x);
    const float r1 = x - __uint_as_float(bx & 0xFFFF0000u);
    const uint32_t b1 = __float_as_uint(r1);
    const float r2 = r1 - __uint_as_float(b1 & 0xFFFF0000u);
    hi = (uint16_t)(bx >> 16);
    mid = (uint16_t)(b1 >> 16);
    lo = bf16_bits_rn(r2);
}

// The network image from the FP32 parameter vector P (layout kOff*): the
// same BF16 roundings as the evaluation copy (W1, W2, W3, W4 rounded to
// nearest BF16, the biases split, b4 unrounded); grid-stride over the
// calling threads (tid of nthreads).
__device__ __forceinline__ void tc_mlp_image(const float *__restrict__ P, TcMlpImage &I, int tid, int nthreads)
{
    uint16_t *w1 = reinterpret_cast<uint16_t *>(I.w1);
    for (int i = tid; i < 64 * 16; i += nthreads) {
        const int n = i >> 4, k = i & 15;
        w1[kmaj_off(64, n, k) / 2] = bf16_bits_rn(k < 15 ? P[kOffW1 + n * kIn + k % 5] : 0.0f);
    }
    // hidden layers: 16-byte units (row n, columns 8j .. 8j+7)
    for (int i = tid; i < 2 * 64 * 8; i += nthreads) {
        const int layer = i >> 9, n = (i >> 3) & 63, j = i & 7;
        const float *W = P + (layer == 0 ? kOffW2 : kOffW3) + n * kHid + 8 * j;
        const uint4 v = make_uint4(pack_bf16(W[0], W[1]), pack_bf16(W[2], W[3]), pack_bf16(W[4], W[5]),
                                   pack_bf16(W[6], W[7]));
        *reinterpret_cast<uint4 *>((layer == 0 ? I.w2 : I.w3) + kmaj_off(64, n, 8 * j)) = v;
    }
    for (int i = tid; i < 3 * 64 * 16; i += nthreads) {
        const int layer = i >> 10, n = (i >> 4) & 63, k = i & 15;
        uint16_t hi, mid, lo;
        split3(P[(layer == 0 ? kOffB1 : (layer == 1 ? kOffB2 : kOffB3)) + n], hi, mid, lo);
        const uint16_t v = k == 0 ? hi : (k == 1 ? mid : (k == 2 ? lo : (uint16_t)0));
        reinterpret_cast<uint16_t *>(I.bias[layer])[kmaj_off(64, n, k) / 2] = v;
    }
    for (int i = tid; i < kTcRows * 16; i += nthreads) {
        const int m = i >> 4, k = i & 15;
        reinterpret_cast<uint16_t *>(I.one)[kmaj_off(kTcRows, m, k) / 2] = k < 3 ? (uint16_t)0x3F80u : (uint16_t)0;
    }
    for (int i = tid; i < 64; i += nthreads) I.w4[i] = __bfloat162float(__float2bfloat16_rn(P[kOffW4 + i]));
    if (tid == 0) {
        I.b4 = P[kOffB4];
        I.pad[0] = I.pad[1] = I.pad[2] = 0.0f;
    }
}

// The network image into shared memory (16-byte copies), the completion
// barrier and the TMEM accumulator.  Called by all threads of the CTA; ends
// with a CTA barrier.
__device__ __forceinline__ void tc_mlp_setup(const MlpDev &w, TcMlpSmem &S)
{
    const int tid = threadIdx.x;
    const uint4 *src = reinterpret_cast<const uint4 *>(w.tc_img);
    uint4 *dst = reinterpret_cast<uint4 *>(&S.img);
    for (int i = tid; i < (int)(sizeof(TcMlpImage) / 16); i += blockDim.x) dst[i] = __ldg(src + i);
    if (tid == 0) {
        tc::mbar_init(&S.mbar, 1);
        tc::fence_mbar_init();
    }
    if (tid < 32) tc::alloc(&S.tmem, kTcCols);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// Release the TMEM accumulator (after a CTA barrier).  When a completion
// wait gave up (`pending`), the last committed MMAs may still be running:
// wait once more, bounded, for the phase of the last commit (`phase` is the
// parity the next wait would use) before the columns are freed.
__device__ __forceinline__ void tc_mlp_teardown(TcMlpSmem &S, unsigned phase = 0u, bool pending = false)
{
    if (pending) tc::mbar_wait(&S.mbar, phase ^ 1u);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) tc::dealloc(S.tmem, kTcCols);
}

// One MMA layer: D = sum over k-steps of A * B, plus the bias step; thread 0
// issues, everyone waits for completion.  nk: K=16 steps of the A operand
// (A columns 16 s .. 16 s + 15 at a + s * (rows / 8) * 256 bytes, B at
// b + s * 8 * 256).
__device__ __forceinline__ bool tc_layer(TcMlpSmem &S, const uint8_t *a, const uint8_t *b, int nk, int layer,
                                         unsigned &phase)
{
    constexpr uint32_t idesc = tc::idesc_bf16(kTcRows, 64);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after();
        const uint32_t sa = tc::saddr(a), sb = tc::saddr(b);
        for (int s = 0; s < nk; ++s)
            tc::mma(S.tmem, tc::desc(sa + s * (kTcRows / 8) * 256, (kTcRows / 8) * 128, 128),
                    tc::desc(sb + s * 8 * 256, 8 * 128, 128), idesc, s > 0);
        tc::mma(S.tmem, tc::desc(tc::saddr(S.img.one), (kTcRows / 8) * 128, 128),
                tc::desc(tc::saddr(S.img.bias[layer]), 8 * 128, 128), idesc, 1);
        tc::commit(&S.mbar);
    }
    const bool ok = tc::mbar_wait(&S.mbar, phase);
    phase ^= 1u;
    tc::fence_after();
    return ok;
}

// Threads per row of a tile: TPR = 1 (128 threads, a whole row each) or
// TPR = 2 (256 threads; warps w and w + 4 read the same TMEM lane quarter,
// w % 4, and take columns 0..31 and 32..63 of its rows): half the serial
// work per thread, for batches too small to fill the GPU with 128-row tiles.
// (threadIdx.x & 96 is the warp's TMEM lane quarter, 32 * (warp % 4).)
template <int TPR> __device__ __forceinline__ int tc_rowid() { return threadIdx.x & (kTcRows - 1); }
template <int TPR> __device__ __forceinline__ int tc_half() { return TPR == 1 ? 0 : (int)(threadIdx.x >> 7); }

// This thread's columns of its row of the accumulator after a layer:
// 64 / TPR FP32 values, from column 64 / TPR * half.
template <int TPR>
__device__ __forceinline__ void tc_row(const TcMlpSmem &S, float (&z)[64 / TPR])
{
    const uint32_t t = S.tmem + ((uint32_t)(threadIdx.x & 96) << 16) + (uint32_t)(tc_half<TPR>() * 32);
    tc::ld32<0>(t, z);
    if (TPR == 1) tc::ld32<(TPR == 1 ? 32 : 0)>(t + 32, z);
    tc::wait_ld();
}

// SiLU of two values with the reciprocal 1 / d, d = 1 + 2^(-z log2 e), by
// Newton-Raphson steps r <- r + r (1 - d r) on the FMA pipe instead of the
// MUFU.  The seed negates the IEEE-754 exponent by an integer subtraction
// from the bit pattern of 2^127 (bits(2^127) - bits(d) ~ bits(1/d) for
// d >= 1) and lies within 12.5 % above 1/d; each step squares the relative
// error, so three take it to 0.125^8 ~ 6e-8.  d is capped at 2^126
// (z < -87, where SiLU is below 1e-36 either way) so the seed stays normal.
__device__ __forceinline__ float2 silu2_nr(float2 z)
{
    constexpr float kNegLog2e = -1.4426950408889634f;
    const float2 m = __fmul2_rn(z, make_float2(kNegLog2e, kNegLog2e));
    float2 d = __fadd2_rn(make_float2(ex2_approx(m.x), ex2_approx(m.y)), make_float2(1.0f, 1.0f));
    d.x = fminf(d.x, 0x1p126f);
    d.y = fminf(d.y, 0x1p126f);
    float2 r = make_float2(__int_as_float(0x7F000000 - __float_as_int(d.x)),
                           __int_as_float(0x7F000000 - __float_as_int(d.y)));
    const float2 nd = __fmul2_rn(d, make_float2(-1.0f, -1.0f));
#pragma unroll
    for (int it = 0; it < 3; ++it) r = __ffma2_rn(r, __ffma2_rn(nd, r, make_float2(1.0f, 1.0f)), r);
    return __fmul2_rn(z, r);
}

// The SiLU pairs of a row (p = 0..31 per layer) are split between the MUFU
// reciprocal and the Newton form so that the MUFU queue and the FMA pipe
// share the work: pair p takes the Newton form when bit (p mod 8) of
// kTcNrMask is set.
#ifndef SPL_TC_NR_MASK
#define SPL_TC_NR_MASK 0x11
#endif
constexpr unsigned kTcNrMask = SPL_TC_NR_MASK;
__device__ __forceinline__ float2 tc_silu2(int p, float2 z)
{
    return ((kTcNrMask >> (p & 7)) & 1u) ? silu2_nr(z) : silu2(z);
}

// SiLU of this thread's columns, rounded to BF16 into its part of the row
// of the A operand of the next layer (and, with SAVE, z and the rounded
// activations to zb / hb, which point at the row).
template <int TPR, bool SAVE>
__device__ __forceinline__ void tc_silu_store(TcMlpSmem &S, const float (&z)[64 / TPR], float *zb, float *hb)
{
    constexpr int NC = 64 / TPR;  // columns of this thread
    const int m = tc_rowid<TPR>(), c0 = NC * tc_half<TPR>();
    if (SAVE) {
#pragma unroll
        for (int k = 0; k < NC; k += 4)
            *reinterpret_cast<float4 *>(zb + c0 + k) = make_float4(z[k], z[k + 1], z[k + 2], z[k + 3]);
    }
#pragma unroll
    for (int j = 0; j < NC / 8; ++j) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 h = tc_silu2(4 * j + q, make_float2(z[8 * j + 2 * q], z[8 * j + 2 * q + 1]));
            w[q] = pack_bf16(h.x, h.y);
        }
        *reinterpret_cast<uint4 *>(S.a2 + kmaj_off(kTcRows, m, c0 + 8 * j)) = make_uint4(w[0], w[1], w[2], w[3]);
        if (SAVE) {
            float4 *d = reinterpret_cast<float4 *>(hb + c0 + 8 * j);
            d[0] = make_float4(__uint_as_float(w[0] << 16), __uint_as_float(w[0] & 0xFFFF0000u),
                               __uint_as_float(w[1] << 16), __uint_as_float(w[1] & 0xFFFF0000u));
            d[1] = make_float4(__uint_as_float(w[2] << 16), __uint_as_float(w[2] & 0xFFFF0000u),
                               __uint_as_float(w[3] << 16), __uint_as_float(w[3] & 0xFFFF0000u));
        }
    }
}

// Optional capture of a tile's activations for training: z1, h1, z2, h2,
// z3, h3 of this thread's row (FP32; h1, h2 as the BF16-rounded values that
// entered the tensor-core layers), 64 values each at row * 64 of the arrays
// (row < 0: nothing is stored).
struct TcSave {
    float *z1, *h1, *z2, *h2, *z3, *h3;
    int row;
};

// f_theta of this thread's row x (5 features) in a tile of 128 rows; every
// thread of the CTA (128 * TPR) calls it, the TPR threads of a row with the
// same x.  Returns false if a tensor-core wait gave up (the output is then
// meaningless).  The output is valid in every thread of the row.  part:
// 2 x 128 floats of shared memory for combining the halves of the output
// layer (TPR = 2; rewritten only after the next tile's first barrier).
// SAVE stores the activations of the row (sv->row >= 0).
template <int TPR, bool SAVE = false>
__device__ __forceinline__ bool tc_mlp_tile(TcMlpSmem &S, const float (&x)[5], float &out, unsigned &phase,
                                            float *part = nullptr, const TcSave *sv = nullptr)
{
    constexpr int NC = 64 / TPR;
    const int m = tc_rowid<TPR>(), half = tc_half<TPR>();
    const bool save = SAVE && sv->row >= 0;
    const size_t ro = SAVE ? (size_t)(sv->row < 0 ? 0 : sv->row) * 64 : 0;
    {
        uint16_t p[16];
#pragma unroll
        for (int e = 0; e < 5; ++e) split3(x[e], p[e], p[5 + e], p[10 + e]);
        p[15] = 0;
        uint32_t v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = (uint32_t)p[2 * q] | ((uint32_t)p[2 * q + 1] << 16);
        if (TPR == 1 || half == 0)
            *reinterpret_cast<uint4 *>(S.a1 + kmaj_off(kTcRows, m, 0)) = make_uint4(v[0], v[1], v[2], v[3]);
        if (TPR == 1 || half == 1)
            *reinterpret_cast<uint4 *>(S.a1 + kmaj_off(kTcRows, m, 8)) = make_uint4(v[4], v[5], v[6], v[7]);
    }
    bool ok = tc_layer(S, S.a1, S.img.w1, 1, 0, phase);
    float z[NC];
    tc_row<TPR>(S, z);
    if (save) tc_silu_store<TPR, true>(S, z, sv->z1 + ro, sv->h1 + ro);
    else tc_silu_store<TPR, false>(S, z, nullptr, nullptr);
    ok &= tc_layer(S, S.a2, S.img.w2, 4, 1, phase);
    tc_row<TPR>(S, z);
    if (save) tc_silu_store<TPR, true>(S, z, sv->z2 + ro, sv->h2 + ro);
    else tc_silu_store<TPR, false>(S, z, nullptr, nullptr);
    ok &= tc_layer(S, S.a2, S.img.w3, 4, 2, phase);
    tc_row<TPR>(S, z);
    const int c0 = NC * half;
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < NC; k += 2) {
        if (save) *reinterpret_cast<float2 *>(sv->z3 + ro + c0 + k) = make_float2(z[k], z[k + 1]);
        const float2 h = tc_silu2(k >> 1, make_float2(z[k], z[k + 1]));
        if (save) *reinterpret_cast<float2 *>(sv->h3 + ro + c0 + k) = h;
        acc = __ffma2_rn(h, make_float2(S.img.w4[c0 + k], S.img.w4[c0 + k + 1]), acc);
    }
    float o = acc.x + acc.y;
    if (TPR == 2) {
        // both threads of the row add the two halves in the same order
        part[half * kTcRows + m] = o;
        __syncthreads();
        o = part[m] + part[kTcRows + m];
    }
    out = o + S.img.b4;
    return ok;
}

}  // namespace spl
