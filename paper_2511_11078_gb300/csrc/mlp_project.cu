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

constexpr int kMlpWarps = 4;
#ifndef SPL_MLP_MIN_BLOCKS
#define SPL_MLP_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for
#endif
constexpr int kMlpThreads = 32 * kMlpWarps;

// most pairs one slab can produce: the initial (N+1)^2 window plus N+1 per
// window shift; a transverse axis crosses at most N+2 knot planes in a slab
// (plus one shift at the slab start when the window position rounds down),
// so at most N+3 shifts per axis.  Rows beyond the capacity are dropped and
// flag an error (never written out of bounds).
template <int N> struct PairCap { static constexpr int value = (N + 1) * (N + 1) + (N + 1) * (2 * N + 6); };

// Per-lane data of the current round (one slab of each lane's ray), which
// the rows of the queue refer to by lane.
struct __align__(16) MlpLaneTab {
    float wc0[32], wc1[32], wc2[32];  // canonical direction of the ray
    float ua[32], ub[32], va[32], vb[32];
    float fa[32], fb[32];  // A_j = IA + fa, B_j = IB + fb on the slab plane
    int base[32];          // address of basis (j, IA - N, IB - N)
    int S1[32], S2[32];    // mirrored strides of the ray's a and b axes
    float yv[32];          // adjoint: the ray's datum
    float acc[32];         // forward: the ray's sum
    int count;
};

// A queue row names one pair in 16 bits: the lane (5 bits) and the pair's
// basis offsets da = la - IA + N, db = lb - IB + N on the lane's slab
// (5 bits each; every window of a slab lies in [IA - N, IA + 2N + 4], so
// they stay below 3N + 5 <= 14).  The features and the coefficient address
// follow from the lane's table:
//   Pa = A_j - la = (N - da) + fa,  Pb = (N - db) + fb,
//   features (wc, ua Pa + ub Pb, va Pa + vb Pb),
//   address base + da S1 + db S2.
struct MlpQueueSink {
    uint16_t *q;
    MlpLaneTab *tab;
    int cap;
    int j, S0, S1, S2;
    int loa, hia, lob, hib;
    int IA, IB;
    int lane;
    bool bad;  // an offset outside 5 bits (not expected; the row is dropped)
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ void slab(int ia, float fa, int ib, float fb, int n)
    {
        IA = ia;
        IB = ib;
        tab->fa[lane] = fa;
        tab->fb[lane] = fb;
        tab->base[lane] = j * S0 + (ia - n) * S1 + (ib - n) * S2;
    }
    __device__ __forceinline__ bool relevant(int a0, int a1, int b0, int b1) const
    {
        return a1 >= loa && a0 <= hia && b1 >= lob && b0 <= hib;
    }
    template <int N> __device__ __forceinline__ void flush_n(int la, int lb, float v)
    {
        if (v > 0.0f && la >= loa && la <= hia && lb >= lob && lb <= hib) {
            const unsigned da = (unsigned)(la - IA + N), db = (unsigned)(lb - IB + N);
            if (da > 31u || db > 31u) {
                bad = true;
                return;
            }
            const int k = atomicAdd(&tab->count, 1);
            if (k < cap) q[k] = (uint16_t)((unsigned)lane | (da << 5) | (db << 10));
        }
    }
};

template <int N> struct MlpSinkN : MlpQueueSink {
    __device__ __forceinline__ void flush(int, int la, int lb, float v) { flush_n<N>(la, lb, v); }
};

// Lane, coefficient address and (Pa, Pb) of queue row e.
template <int N>
__device__ __forceinline__ void decode_row(const MlpLaneTab &T, unsigned e, int &l, int &addr, float &Pa, float &Pb)
{
    l = (int)(e & 31u);
    const int da = (int)((e >> 5) & 31u), db = (int)(e >> 10);
    addr = T.base[l] + da * T.S1[l] + db * T.S2[l];
    Pa = (float)(N - da) + T.fa[l];
    Pb = (float)(N - db) + T.fb[l];
}

template <int N> constexpr int mlp_queue_bytes() { return (32 * PairCap<N>::value * 2 + 15) / 16 * 16; }
template <int N> constexpr size_t mlp_views_smem()
{
    return sizeof(MlpSmem) + (size_t)kMlpWarps * (sizeof(MlpLaneTab) + mlp_queue_bytes<N>());
}

// ADJ = false: y = A_theta c ; ADJ = true: c += A_theta^T y (c zeroed by the host)
template <int N, bool ADJ>
__global__ void __launch_bounds__(kMlpThreads, SPL_MLP_MIN_BLOCKS) k_mlp_views(DevGeom g, MlpDev wts, const float *__restrict__ cin,
                                                              float *__restrict__ yout, const float *__restrict__ yin,
                                                              float *__restrict__ cout, QuadRule qr)
{
    extern __shared__ __align__(16) unsigned char smem[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem);
    constexpr int cap = 32 * PairCap<N>::value;
    mlp_load_smem(wts, S);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g4 = lane >> 2, t4 = lane & 3;
    unsigned char *wbase = smem + sizeof(MlpSmem) + (size_t)wid * (sizeof(MlpLaneTab) + mlp_queue_bytes<N>());
    MlpLaneTab &T = *reinterpret_cast<MlpLaneTab *>(wbase);
    uint16_t *q = reinterpret_cast<uint16_t *>(wbase + sizeof(MlpLaneTab));
    const int iu = blockIdx.x * 8 + (lane & 7), iv = blockIdx.y * (4 * kMlpWarps) + wid * 4 + (lane >> 3);
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
        rs.S[0] = rs.S[1] = rs.S[2] = 0;
    }
    T.wc0[lane] = mr.wc[0];
    T.wc1[lane] = mr.wc[1];
    T.wc2[lane] = mr.wc[2];
    T.ua[lane] = mr.ua;
    T.ub[lane] = mr.ub;
    T.va[lane] = mr.va;
    T.vb[lane] = mr.vb;
    T.S1[lane] = rs.S[1];
    T.S2[lane] = rs.S[2];
    T.acc[lane] = 0.0f;
    T.yv[lane] = yr;
    if (lane == 0) T.count = 0;
    __syncthreads();  // weights in shared memory
    const int nslab = rs.j1 - rs.j0 + 1;
    const int rounds = __reduce_max_sync(0xffffffffu, nslab > 0 ? nslab : 0);
    bool ok = true;
    for (int round = 0; round < rounds; ++round) {
        if (round < nslab) {
            MlpSinkN<N> sk;
            sk.q = q;
            sk.tab = &T;
            sk.cap = cap;
            sk.j = rs.j0 + round;
            sk.S0 = rs.S[0];
            sk.S1 = rs.S[1];
            sk.S2 = rs.S[2];
            sk.loa = rs.lo[1];
            sk.hia = rs.hi[1];
            sk.lob = rs.lo[2];
            sk.hib = rs.hi[2];
            sk.IA = sk.IB = 0;
            sk.lane = lane;
            sk.bad = false;
            ok &= slab_pairs<N, MlpSinkN<N>>(rs, sk.j, qr, sk);
            ok &= !sk.bad;
        }
        __syncwarp();
        int n = T.count;
        if (n > cap) {
            ok = false;
            n = cap;
        }
        for (int base = 0; base < n; base += 16) {
            float x[2][5];
            float cv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = base + g4 + 8 * h;
                cv[h] = 0.0f;
#pragma unroll
                for (int i = 0; i < 5; ++i) x[h][i] = 0.0f;
                if (r < n) {
                    int l, addr;
                    float Pa, Pb;
                    decode_row<N>(T, q[r], l, addr, Pa, Pb);
                    if (!ADJ) cv[h] = __ldg(cin + addr);
                    x[h][0] = T.wc0[l];
                    x[h][1] = T.wc1[l];
                    x[h][2] = T.wc2[l];
                    x[h][3] = fmaf(T.ua[l], Pa, T.ub[l] * Pb);
                    x[h][4] = fmaf(T.va[l], Pa, T.vb[l] * Pb);
                }
            }
            float o[2];
            mlp_tile16<false>(S, x[0], x[1], o[0], o[1]);
            if (t4 == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = base + g4 + 8 * h;
                    if (r >= n) continue;
                    int l, addr;
                    float Pa, Pb;
                    decode_row<N>(T, q[r], l, addr, Pa, Pb);
                    if (ADJ) atomicAdd(cout + addr, T.yv[l] * o[h]);
                    else atomicAdd(&T.acc[l], cv[h] * o[h]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) T.count = 0;
        __syncwarp();
    }
    if (!ok) atomicOr(g.err, 1);
    if (!ADJ && valid) {
        __syncwarp();
        yout[ray] = T.acc[lane];
    }
}

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
    dim3 grid((dg.nu + 7) / 8, (dg.nv + 4 * kMlpWarps - 1) / (4 * kMlpWarps), dg.n_views);
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
