// mlp_project.cu -- forward projection and adjoint with the learned
// footprint f_theta in place of the exact one (Algorithm 2 with f_theta*).
//
// A CTA owns 128 rays (an 8 x 16 detector tile).  It walks the rays' slabs
// in lock-step rounds: in each round every thread sweeps one slab of its ray
// in pair-enumeration mode (the same dominant-axis slab march and window as
// the exact path, so the pair set is the exact support of every basis --
// f_theta is kept only where the ray meets the basis) and appends one 16-bit
// row per pair to the CTA's queue in shared memory.  The CTA then drains the
// queue in tiles of 128 rows through the tcgen05 network (one row per
// thread, accumulator in TMEM) and accumulates c * f_theta per ray (forward,
// shared-memory atomics) or y_r * f_theta per coefficient (adjoint, float
// atomics in global memory).
#include "spl_tc.cuh"

namespace spl {

constexpr int kMlpThreads = kTcRows;

// most pairs one slab can produce: the initial (N+1)^2 window plus N+1 per
// window shift; a transverse axis crosses at most N+2 knot planes in a slab
// (plus one shift at the slab start when the window position rounds down),
// so at most N+3 shifts per axis.  Rows beyond the capacity are dropped and
// flag an error (never written out of bounds).
template <int N> struct PairCap { static constexpr int value = (N + 1) * (N + 1) + (N + 1) * (2 * N + 6); };

// Per-ray data of the current round (one slab of each thread's ray), which
// the rows of the queue refer to by ray.
struct __align__(16) MlpRayRec {
    float4 a;  // canonical direction wc0, wc1, wc2; ua
    float4 b;  // ub, va, vb; fa (A_j = IA + fa on the slab plane)
    int4 c;    // fb (float bits; B_j = IB + fb); address of basis (j, IA - N, IB - N);
               // mirrored strides S1, S2 of the ray's a and b axes
};
struct __align__(16) MlpRayTab {
    MlpRayRec rec[kMlpThreads];
    float yv[kMlpThreads];   // adjoint: the ray's datum
    float acc[kMlpThreads];  // forward: the ray's sum
    int count;               // rows in the queue
    int rounds;              // slabs of the longest ray of the CTA
};

// A queue row names one pair in 15 bits: the ray (7 bits) and the pair's
// basis offsets da = la - IA + N, db = lb - IB + N on the ray's slab
// (4 bits each; every window of a slab lies in [IA - N, IA + 2N + 4], so
// they stay below 3N + 5 <= 14).  The features and the coefficient address
// follow from the ray's table entry:
//   Pa = A_j - la = (N - da) + fa,  Pb = (N - db) + fb,
//   features (wc, ua Pa + ub Pb, va Pa + vb Pb),
//   address base + da S1 + db S2.
struct MlpQueueSink {
    uint16_t *q;
    MlpRayTab *tab;
    int cap;
    int j, S0, S1, S2;
    int loa, hia, lob, hib;
    int IA, IB;
    int ray;
    bool bad;  // an offset outside 4 bits (not expected; the row is dropped)
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ void slab(int ia, float fa, int ib, float fb, int n)
    {
        IA = ia;
        IB = ib;
        tab->rec[ray].b.w = fa;
        tab->rec[ray].c.x = __float_as_int(fb);
        tab->rec[ray].c.y = j * S0 + (ia - n) * S1 + (ib - n) * S2;
    }
    __device__ __forceinline__ bool relevant(int a0, int a1, int b0, int b1) const
    {
        return a1 >= loa && a0 <= hia && b1 >= lob && b0 <= hib;
    }
    template <int N> __device__ __forceinline__ void flush_n(int la, int lb, float v)
    {
        if (v > 0.0f && la >= loa && la <= hia && lb >= lob && lb <= hib) {
            const unsigned da = (unsigned)(la - IA + N), db = (unsigned)(lb - IB + N);
            if (da > 15u || db > 15u) {
                bad = true;
                return;
            }
            const int k = atomicAdd(&tab->count, 1);
            if (k < cap) q[k] = (uint16_t)((unsigned)ray | (da << 7) | (db << 11));
        }
    }
};

template <int N> struct MlpSinkN : MlpQueueSink {
    __device__ __forceinline__ void flush(int, int la, int lb, float v) { flush_n<N>(la, lb, v); }
};

// Ray, coefficient address and features of queue row e.
template <int N>
__device__ __forceinline__ void decode_row(const MlpRayTab &T, unsigned e, int &l, int &addr, float (&x)[5])
{
    l = (int)(e & 127u);
    const int da = (int)((e >> 7) & 15u), db = (int)(e >> 11);
    const float4 A = T.rec[l].a, B = T.rec[l].b;
    const int4 C = T.rec[l].c;
    addr = C.y + da * C.z + db * C.w;
    const float Pa = (float)(N - da) + B.w, Pb = (float)(N - db) + __int_as_float(C.x);
    x[0] = A.x;
    x[1] = A.y;
    x[2] = A.z;
    x[3] = fmaf(A.w, Pa, B.x * Pb);
    x[4] = fmaf(B.y, Pa, B.z * Pb);
}

template <int N> constexpr int mlp_queue_bytes() { return (kMlpThreads * PairCap<N>::value * 2 + 15) / 16 * 16; }
template <int N> constexpr size_t mlp_views_smem()
{
    return sizeof(TcMlpSmem) + sizeof(MlpRayTab) + (size_t)mlp_queue_bytes<N>();
}

// ADJ = false: y = A_theta c ; ADJ = true: c += A_theta^T y (c zeroed by the host)
template <int N, bool ADJ>
__global__ void __launch_bounds__(kMlpThreads, 3) k_mlp_views(DevGeom g, MlpDev wts, const float *__restrict__ cin,
                                                           float *__restrict__ yout, const float *__restrict__ yin,
                                                           float *__restrict__ cout, QuadRule qr)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    TcMlpSmem &S = *reinterpret_cast<TcMlpSmem *>(smem);
    MlpRayTab &T = *reinterpret_cast<MlpRayTab *>(smem + sizeof(TcMlpSmem));
    uint16_t *q = reinterpret_cast<uint16_t *>(smem + sizeof(TcMlpSmem) + sizeof(MlpRayTab));
    constexpr int cap = kMlpThreads * PairCap<N>::value;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        T.count = 0;
        T.rounds = 0;
    }
    tc_mlp_setup(wts, S);  // ends with a CTA barrier
    const int iu = blockIdx.x * 8 + (lane & 7), iv = blockIdx.y * 16 + wid * 4 + (lane >> 3);
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
    T.rec[tid].a = make_float4(mr.wc[0], mr.wc[1], mr.wc[2], mr.ua);
    T.rec[tid].b = make_float4(mr.ub, mr.va, mr.vb, 0.0f);
    T.rec[tid].c = make_int4(0, 0, rs.S[1], rs.S[2]);
    T.acc[tid] = 0.0f;
    T.yv[tid] = yr;
    const int nslab = rs.j1 - rs.j0 + 1;
    if (nslab > 0) atomicMax(&T.rounds, nslab);
    __syncthreads();
    const int rounds = T.rounds;
    unsigned phase = 0;
    bool ok = true, stop = false, timeout = false;
    for (int round = 0; round < rounds && !stop; ++round) {
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
            sk.ray = tid;
            sk.bad = false;
            ok &= slab_pairs<N, MlpSinkN<N>>(rs, sk.j, qr, sk);
            ok &= !sk.bad;
        }
        __syncthreads();
        int n = T.count;
        if (n > cap) {
            ok = false;
            n = cap;
        }
        for (int base = 0; base < n; base += kMlpThreads) {
            const int r = base + tid;
            float x[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            float cv = 0.0f;
            int l = 0, addr = 0;
            if (r < n) {
                decode_row<N>(T, q[r], l, addr, x);
                if (!ADJ) cv = __ldg(cin + addr);
            }
            float o;
            const bool tok = tc_mlp_tile<1>(S, x, o, phase);
            if (__syncthreads_or(!tok)) {  // a tensor-core wait gave up (not expected)
                timeout = true;
                stop = true;
                break;
            }
            if (r < n) {
                if (ADJ) atomicAdd(cout + addr, T.yv[l] * o);
                else atomicAdd(&T.acc[l], cv * o);
            }
        }
        __syncthreads();  // queue drained
        if (tid == 0) T.count = 0;
        __syncthreads();
    }
    if (!ok) atomicOr(g.err, kErrStepCap);
    if (timeout && tid == 0) atomicOr(g.err, kErrTimeout);
    if (!ADJ && valid) yout[ray] = timeout ? __int_as_float(0x7FC00000) : T.acc[tid];
    tc_mlp_teardown(S, phase, timeout);
}

template <int N, bool ADJ>
static spl_status launch_mlp_views(const spl_geometry *g, const spl_mlp *m, const float *cin, float *yout,
                                   const float *yin, float *cout, cudaStream_t st)
{
    const DevGeom &dg = g->dev;
    if (dg.n_rays == 0) return SPL_OK;
    const size_t sm = mlp_views_smem<N>();
    {
        spl_status s = smem_attr_once((const void *)k_mlp_views<N, ADJ>, (int)sm, "mlp smem attribute");
        if (s != SPL_OK) return s;
    }
    dim3 grid((dg.nu + 7) / 8, (dg.nv + 15) / 16, dg.n_views);
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
