// mlp_project.cu -- forward projection and adjoint with the learned
// footprint f_theta in place of the exact one (Algorithm 2 with f_theta*).
//
// A warp owns 32 rays (an 8 x 4 detector sub-tile).  The warp walks the
// rays' slabs in lock-step rounds: in each round every lane sweeps one slab
// of its ray in pair-enumeration mode (the same dominant-axis slab march and
// window as the exact path, so the pair set is the exact support of every
// basis -- f_theta is kept only where the ray meets the basis), and appends
// one row per pair to a per-warp queue in shared memory: the two ray-
// dependent features (the canonical direction is per ray) and the
// coefficient (forward) or its address (adjoint).  The warp then drains the
// queue in 16-row tiles through the BF16 tensor-core MLP and accumulates
// c * f_theta per ray (forward) or y_r * f_theta per coefficient with float
// atomics (adjoint).
#include "spl_mlp.cuh"

namespace spl {

constexpr int kMlpWarps = 2;
constexpr int kMlpThreads = 32 * kMlpWarps;

// most pairs one slab can produce: the initial (N+1)^2 window plus N+1 per
// window shift; a transverse axis crosses at most N+2 knot planes in a slab
// (plus one shift at the slab start when the window position rounds down),
// so at most N+3 shifts per axis.  Rows beyond the capacity are dropped and
// flag an error (never written out of bounds).
template <int N> struct PairCap { static constexpr int value = (N + 1) * (N + 1) + (N + 1) * (2 * N + 6); };

struct MlpWarpQueue {
    float f3, f4;
    int val;   // forward: coefficient (float bits); adjoint: coefficient index
    int lane;  // lane whose ray produced the row
};

struct MlpQueueSink {
    MlpWarpQueue *q;
    int *count;
    int cap;
    const float *__restrict__ c;
    int S0, S1, S2;
    int loa, hia, lob, hib;
    float ua, ub, va, vb;
    int IA, IB;
    float fa, fb;
    int lane;
    bool adj;
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ void slab(int ia, float fa_, int ib, float fb_, int)
    {
        IA = ia;
        fa = fa_;
        IB = ib;
        fb = fb_;
    }
    __device__ __forceinline__ bool relevant(int a0, int a1, int b0, int b1) const
    {
        return a1 >= loa && a0 <= hia && b1 >= lob && b0 <= hib;
    }
    __device__ __forceinline__ void flush(int j, int la, int lb, float v)
    {
        if (v > 0.0f && la >= loa && la <= hia && lb >= lob && lb <= hib) {
            const float Pa = (float)(IA - la) + fa, Pb = (float)(IB - lb) + fb;
            const int addr = j * S0 + la * S1 + lb * S2;
            const int k = atomicAdd(count, 1);
            if (k < cap) {
                MlpWarpQueue e;
                e.f3 = fmaf(ua, Pa, ub * Pb);
                e.f4 = fmaf(va, Pa, vb * Pb);
                e.val = adj ? addr : __float_as_int(__ldg(c + addr));
                e.lane = lane;
                q[k] = e;
            }
        }
    }
};

// ADJ = false: y = A_theta c ; ADJ = true: c += A_theta^T y (c zeroed by the host)
template <int N, bool ADJ>
__global__ void __launch_bounds__(kMlpThreads) k_mlp_views(DevGeom g, MlpDev wts, const float *__restrict__ cin,
                                                           float *__restrict__ yout, const float *__restrict__ yin,
                                                           float *__restrict__ cout, QuadRule qr)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
    constexpr int cap = 32 * PairCap<N>::value;
    MlpWarpQueue *queues = reinterpret_cast<MlpWarpQueue *>(smem + sizeof(MlpSmem));
    __shared__ float wc_s[kMlpWarps][32][3];
    __shared__ float acc_s[kMlpWarps][32];
    __shared__ float yv_s[kMlpWarps][32];
    __shared__ int count_s[kMlpWarps];
    mlp_load_smem(wts, S);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g4 = lane >> 2, t4 = lane & 3;
    MlpWarpQueue *q = queues + wid * cap;
    const int iu = blockIdx.x * 8 + (lane & 7), iv = blockIdx.y * 8 + wid * 4 + (lane >> 3);
    const int k = blockIdx.z;
    const bool valid = iu < g.nu && iv < g.nv;
    const long long ray = ((long long)k * g.nv + (valid ? iv : 0)) * g.nu + (valid ? iu : 0);
    RaySetup rs;
    MlpRay mr;
    bool live = false;
    float yr = 0.0f;
    if (valid) {
        if (ADJ) yr = __ldg(yin + ray);
        double s[3], w[3];
        view_ray(g, k, iu, iv, s, w);
        live = (!ADJ || yr != 0.0f) && view_setup<N>(g, grid_of(g), k, iu, iv, rs);
        if (live) {
            int ax[3] = {rs.ax[0], rs.ax[1], rs.ax[2]};
            mlp_ray_setup(N, w, ax, mr);
        }
    }
    if (!live) {
        rs.j0 = 0;
        rs.j1 = -1;
        mr.wc[0] = mr.wc[1] = mr.wc[2] = 0.0f;
        mr.ua = mr.ub = mr.va = mr.vb = 0.0f;
    }
    wc_s[wid][lane][0] = mr.wc[0];
    wc_s[wid][lane][1] = mr.wc[1];
    wc_s[wid][lane][2] = mr.wc[2];
    acc_s[wid][lane] = 0.0f;
    yv_s[wid][lane] = yr;
    if (lane == 0) count_s[wid] = 0;
    __syncthreads();  // weights in shared memory
    const int nslab = rs.j1 - rs.j0 + 1;
    const int rounds = __reduce_max_sync(0xffffffffu, nslab > 0 ? nslab : 0);
    bool ok = true;
    for (int round = 0; round < rounds; ++round) {
        if (round < nslab) {
            MlpQueueSink sk{q, &count_s[wid], cap, cin, rs.S[0], rs.S[1], rs.S[2], rs.lo[1], rs.hi[1], rs.lo[2], rs.hi[2],
                            mr.ua, mr.ub, mr.va, mr.vb, 0, 0, 0.0f, 0.0f, lane, ADJ};
            ok &= slab_pairs<N, MlpQueueSink>(rs, rs.j0 + round, qr, sk);
        }
        __syncwarp();
        int n = count_s[wid];
        if (n > cap) {
            ok = false;
            n = cap;
        }
        for (int base = 0; base < n; base += 16) {
            float x[2][5];
            MlpWarpQueue e[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = base + g4 + 8 * h;
                if (r < n) {
                    e[h] = q[r];
                    const int ln = e[h].lane;
                    x[h][0] = wc_s[wid][ln][0];
                    x[h][1] = wc_s[wid][ln][1];
                    x[h][2] = wc_s[wid][ln][2];
                    x[h][3] = e[h].f3;
                    x[h][4] = e[h].f4;
                } else {
                    e[h].lane = -1;
#pragma unroll
                    for (int i = 0; i < 5; ++i) x[h][i] = 0.0f;
                }
            }
            float o[2];
            mlp_tile16<false>(S, x[0], x[1], o[0], o[1]);
            if (t4 == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (e[h].lane < 0) continue;
                    const int ln = e[h].lane;
                    if (ADJ) atomicAdd(cout + e[h].val, yv_s[wid][ln] * o[h]);
                    else atomicAdd(&acc_s[wid][ln], __int_as_float(e[h].val) * o[h]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) count_s[wid] = 0;
        __syncwarp();
    }
    if (!ok) atomicOr(g.err, 1);
    if (!ADJ && valid) {
        __syncwarp();
        yout[ray] = acc_s[wid][lane];
    }
}

template <int N> constexpr size_t mlp_views_smem() { return sizeof(MlpSmem) + (size_t)kMlpWarps * 32 * PairCap<N>::value * sizeof(MlpWarpQueue); }

template <int N, bool ADJ>
static spl_status launch_mlp_views(const spl_geometry *g, const spl_mlp *m, const float *cin, float *yout,
                                   const float *yin, float *cout, cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    if (dg.n_rays == 0) return SPL_OK;
    const size_t sm = mlp_views_smem<N>();
    static bool attr_done = false;
    if (!attr_done) {
        spl_status s = cuda_check(cudaFuncSetAttribute(k_mlp_views<N, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)sm),
                                  "mlp smem attribute");
        if (s != SPL_OK) return s;
        attr_done = true;
    }
    dim3 grid((dg.nu + 7) / 8, (dg.nv + 7) / 8, dg.n_views);
    k_mlp_views<N, ADJ><<<grid, kMlpThreads, sm, st>>>(dg, mlp_dev(m), cin, yout, yin, cout, quad_rule(N));
    return cuda_check(cudaGetLastError(), "mlp projector launch");
}

spl_status forward_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st)
{
    switch (b->degree) {
    case 0: return launch_mlp_views<0, false>(g, b->mlp, c, y, nullptr, nullptr, st);
    case 1: return launch_mlp_views<1, false>(g, b->mlp, c, y, nullptr, nullptr, st);
    case 2: return launch_mlp_views<2, false>(g, b->mlp, c, y, nullptr, nullptr, st);
    default: return launch_mlp_views<3, false>(g, b->mlp, c, y, nullptr, nullptr, st);
    }
}

spl_status adjoint_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st)
{
    const long long nc = (long long)g->dev.n[0] * g->dev.n[1] * g->dev.n[2];
    spl_status s = cuda_check(cudaMemsetAsync(c, 0, nc * sizeof(float), st), "adjoint clear");
    if (s != SPL_OK) return s;
    switch (b->degree) {
    case 0: return launch_mlp_views<0, true>(g, b->mlp, nullptr, nullptr, y, c, st);
    case 1: return launch_mlp_views<1, true>(g, b->mlp, nullptr, nullptr, y, c, st);
    case 2: return launch_mlp_views<2, true>(g, b->mlp, nullptr, nullptr, y, c, st);
    default: return launch_mlp_views<3, true>(g, b->mlp, nullptr, nullptr, y, c, st);
    }
}

}  // namespace spl
