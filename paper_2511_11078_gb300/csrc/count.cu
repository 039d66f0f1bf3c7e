// count.cu -- the number of contributions of Eq. 4: (ray, basis) pairs
// whose line meets the open support cube [k - W, k + W]^3 of the basis in a
// segment of positive length (W = (n+1)/2).
//
// The count is index work that floating point decides, so it is decided
// here in the same precision and with the same operations as the plain
// definition: each ray is rebuilt from the caller's FP64 pose arrays (pixel
// centre det_center + a det_u + b det_v, direction over its norm), and along
// each axis e the line is inside the support slab of index k for t in
// (lo_e(k), hi_e(k)), the sorted pair of (-W - p)/w_e and (W - p)/w_e with
// p = s_e - (origin_e + k); a pair counts when max_e lo_e < min_e hi_e.  An
// axis with w_e = 0 admits the indices whose B-spline value at p is
// positive, with the interval (-inf, inf).  Every product, sum, quotient and
// square root is rounded separately (no fused multiply-add), so the
// decisions are those of the same formulas evaluated in FP64 anywhere.
//
// Enumeration: one thread per ray sweeps the indices of its dominant axis d
// in the order of increasing t.  The intervals of each other axis are
// monotone in t along their own traversal order, so the indices whose
// intervals overlap a slab's interval form a contiguous run: a queue holds
// that run (pushed when its lower end passes below the slab's upper end,
// popped when its upper end falls to the slab's lower end), and each
// interval is computed once per ray.  The starting indices are estimated and
// then moved back until every skipped index is verified to lie wholly
// before the ray's first relevant slab.
#include "spl_host.h"

namespace spl {

namespace {

constexpr int kQueue = 16;         // per transverse axis; at most 2n + 3 intervals overlap a slab
constexpr int kCountThreads = 64;

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// the ray of index r: s, and w = dir / |dir| with |dir|^2 = (d0 d0 + d1 d1) + d2 d2
__device__ void exact_ray(const DevGeom &g, long long r, double (&s)[3], double (&w)[3])
{
    double dir[3];
    if (g.kind == SPL_RAYS) {
        const double *R = g.raw + 6 * r;
        for (int e = 0; e < 3; ++e) {
            dir[e] = R[e];
            s[e] = R[3 + e];
        }
    } else {
        const long long per = (long long)g.nu * g.nv;
        const int v = (int)(r / per);
        const long long rem = r - (long long)v * per;
        const int iv = (int)(rem / g.nu), iu = (int)(rem - (long long)iv * g.nu);
        const double a = (double)iu - 0.5 * (double)(g.nu - 1), b = (double)iv - 0.5 * (double)(g.nv - 1);
        const double *P = g.raw + 12 * (long long)v;  // direction or source, detector centre, det_u, det_v
        for (int e = 0; e < 3; ++e) {
            const double q = dadd(dadd(P[3 + e], dmul(a, P[6 + e])), dmul(b, P[9 + e]));
            if (g.kind == SPL_PARALLEL) {
                dir[e] = P[e];
                s[e] = q;
            } else {
                dir[e] = dsub(q, P[e]);
                s[e] = P[e];
            }
        }
    }
    const double nrm = __dsqrt_rn(dadd(dadd(dmul(dir[0], dir[0]), dmul(dir[1], dir[1])), dmul(dir[2], dir[2])));
    for (int e = 0; e < 3; ++e) w[e] = __ddiv_rn(dir[e], nrm);
}

// beta^n(p) > 0 by the truncated-power sum (1/n!) sum_k (-1)^k C(n+1,k)
// (-|p| + W - k)_+^n, in that order of operations (degree 0: the half-open
// box [-1/2, 1/2))
__device__ bool bspline_positive(int n, double p)
{
    if (n == 0) return p >= -0.5 && p < 0.5;
    const double W = 0.5 * (n + 1);
    const double xa = -fabs(p);
    double sum = 0.0, binom = 1.0, fact = 1.0;
    for (int i = 2; i <= n; ++i) fact = dmul(fact, (double)i);
    for (int k = 0; k <= n + 1; ++k) {
        const double u = dsub(dadd(xa, W), (double)k);
        if (u > 0.0) {
            double pw = 1.0;
            for (int i = 0; i < n; ++i) pw = dmul(pw, u);
            sum = dadd(sum, dmul((k & 1) ? -binom : binom, pw));
        }
        binom = __ddiv_rn(dmul(binom, (double)(n + 1 - k)), (double)(k + 1));
    }
    return __ddiv_rn(sum, fact) > 0.0;
}

struct Axis {
    double s, w, org, W;
    int n;        // indices 0 .. n-1
    int step;     // +1 or -1: the traversal order of increasing t
    __device__ __forceinline__ void iv(int k, double &lo, double &hi) const
    {
        const double p = dsub(s, dadd(org, (double)k));
        const double t1 = __ddiv_rn(dsub(-W, p), w), t2 = __ddiv_rn(dsub(W, p), w);
        lo = t1 < t2 ? t1 : t2;
        hi = t1 < t2 ? t2 : t1;
    }
    __device__ __forceinline__ int first() const { return step > 0 ? 0 : n - 1; }
    __device__ __forceinline__ bool inside(int k) const { return k >= 0 && k < n; }
    // the first index (in traversal order) whose interval may end after t:
    // an estimate moved back while the index before it still ends after t,
    // so every index skipped ends at or before t
    __device__ int start_after(double t) const
    {
        // hi(k) ~ (W - s + org + k) / w for w > 0, (-W - s + org + k) / w for w < 0
        const double kr = step > 0 ? t * w - W + s - org : t * w + W + s - org;
        double ke = step > 0 ? floor(kr) - 2.0 : ceil(kr) + 2.0;
        if (!(ke > -1.0)) ke = -1.0;
        if (!(ke < (double)n)) ke = (double)n;
        int k = (int)ke;
        if (k < 0) k = step > 0 ? 0 : -1;
        if (k > n - 1) k = step > 0 ? n : n - 1;
        // move back while the previous index in traversal order ends after t
        for (int it = 0; it < 4 * n + 8; ++it) {
            const int kp = k - step;
            if (!inside(kp)) break;
            double lo, hi;
            iv(kp, lo, hi);
            if (!(hi > t)) break;
            k = kp;
        }
        return k;
    }
};

// An FP64 value as an integer with the same order (-0 and +0 equal): the
// comparisons of the sweep then run on the integer units (GB300's FP64
// throughput is a small fraction of its integer throughput).
__device__ __forceinline__ long long okey(double x)
{
    const long long b = __double_as_longlong(__dadd_rn(x, 0.0));  // -0 -> +0
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}

// a queue of the intervals of one transverse axis (a contiguous run of its
// indices in traversal order), as order keys; storage in shared memory
struct Queue {
    long long *lo, *hi;  // kQueue entries each, strided by the block size
    int head, len;
    int next;            // next index to consider (traversal order)
    bool flat;           // w = 0: a fixed set of indices with (-inf, inf)
    __device__ __forceinline__ long long &L(int i) { return lo[((head + i) & (kQueue - 1)) * kCountThreads]; }
    __device__ __forceinline__ long long &H(int i) { return hi[((head + i) & (kQueue - 1)) * kCountThreads]; }
};

// prepare an axis' queue: flat axes get their admitted indices; others
// start at the first index that may end after t0
__device__ bool queue_init(Queue &q, const Axis &ax, int deg, double t0, long long *slo, long long *shi)
{
    q.lo = slo;
    q.hi = shi;
    q.head = 0;
    q.len = 0;
    q.flat = ax.w == 0.0;
    if (q.flat) {
        for (int k = 0; k < ax.n; ++k) {
            const double p = dsub(ax.s, dadd(ax.org, (double)k));
            if (!(fabs(p) < ax.W + 1.0)) continue;
            if (!bspline_positive(deg, p)) continue;
            if (q.len == kQueue) return false;
            q.L(q.len) = okey(-INFINITY);
            q.H(q.len) = okey(INFINITY);
            ++q.len;
        }
        q.next = -1;
        return true;
    }
    q.next = ax.start_after(t0);
    return true;
}

// bring the queue to the run of intervals overlapping (Ld, Hd): push while
// the next interval starts before Hd, pop while the first ends at or before Ld
__device__ bool queue_advance(Queue &q, const Axis &ax, long long Ld, long long Hd)
{
    if (q.flat) return true;
    for (int it = 0; it < 2 * ax.n + 8; ++it) {
        if (!ax.inside(q.next)) break;
        double lo, hi;
        ax.iv(q.next, lo, hi);
        const long long kl = okey(lo);
        if (!(kl < Hd)) break;
        if (q.len == kQueue) {
            // the front must end before the slab for the run to exceed
            // the capacity; drop it if it does, otherwise give up
            if (!(q.H(0) <= Ld)) return false;
            q.head = (q.head + 1) & (kQueue - 1);
            --q.len;
        }
        q.L(q.len) = kl;
        q.H(q.len) = okey(hi);
        ++q.len;
        q.next += ax.step;
    }
    while (q.len > 0 && q.H(0) <= Ld) {
        q.head = (q.head + 1) & (kQueue - 1);
        --q.len;
    }
    return true;
}

template <int DEG>
__device__ unsigned long long count_ray(const DevGeom &g, const double (&s)[3], const double (&w)[3], bool &ok,
                                        long long *slo, long long *shi)
{
    constexpr double W = 0.5 * (DEG + 1);
    // dominant axis d (any axis with w != 0 would do), the others a, b
    int d = 0;
    if (fabs(w[1]) > fabs(w[d])) d = 1;
    if (fabs(w[2]) > fabs(w[d])) d = 2;
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
    Axis A[3];
    for (int e = 0; e < 3; ++e) {
        A[e].s = s[e];
        A[e].w = w[e];
        A[e].org = g.org[e];
        A[e].W = W;
        A[e].n = g.n[e];
        A[e].step = w[e] < 0.0 ? -1 : 1;
    }
    // the earliest t any pair can start: no interval of a (or b) begins
    // before that of its first index in traversal order
    double t0 = -INFINITY;
    for (int e : {a, b}) {
        if (w[e] == 0.0) continue;
        double lo, hi;
        A[e].iv(A[e].first(), lo, hi);
        t0 = lo > t0 ? lo : t0;
    }
    Queue qa, qb;
    if (!queue_init(qa, A[a], DEG, t0, slo, shi) || !queue_init(qb, A[b], DEG, t0, slo + kQueue * kCountThreads,
                                                                  shi + kQueue * kCountThreads)) {
        ok = false;
        return 0;
    }
    if ((qa.flat && qa.len == 0) || (qb.flat && qb.len == 0)) return 0;
    unsigned long long count = 0;
    int kd = A[d].start_after(t0);
    for (int it = 0; it < A[d].n + 1 && A[d].inside(kd); ++it, kd += A[d].step) {
        double ld, hd;
        A[d].iv(kd, ld, hd);
        const long long Ld = okey(ld), Hd = okey(hd);
        if (!queue_advance(qa, A[a], Ld, Hd) || !queue_advance(qb, A[b], Ld, Hd)) {
            ok = false;
            return count;
        }
        // nothing left to meet: a transverse axis exhausted past this slab
        if ((qa.len == 0 && !qa.flat && !A[a].inside(qa.next)) || (qb.len == 0 && !qb.flat && !A[b].inside(qb.next)))
            break;
        // For each a of the run, (L1, H1) = its interval within the slab's;
        // b counts when lo_b < H1 and hi_b > L1.  Both ends of the b
        // intervals increase along the run, so the b with lo_b < H1 form a
        // prefix, those with hi_b <= L1 a shorter prefix, and the count is
        // the difference; L1 and H1 increase with a, so both prefix ends
        // only move forward.
        int jl = 0, jh = 0;
        for (int i = 0; i < qa.len; ++i) {
            const long long la = qa.L(i), ha = qa.H(i);
            const long long L1 = la > Ld ? la : Ld, H1 = ha < Hd ? ha : Hd;
            if (!(H1 > L1)) continue;
            while (jl < qb.len && qb.L(jl) < H1) ++jl;
            while (jh < qb.len && qb.H(jh) <= L1) ++jh;
            count += jl > jh ? (unsigned long long)(jl - jh) : 0ull;
        }
    }
    return count;
}

// per_ray (nullable): the count of each ray
template <int DEG>
__global__ void __launch_bounds__(kCountThreads) k_count_exact(DevGeom g, unsigned long long *total,
                                                               unsigned *per_ray)
{
    __shared__ long long qlo[2 * kQueue * kCountThreads], qhi[2 * kQueue * kCountThreads];
    const long long r = (long long)blockIdx.x * kCountThreads + threadIdx.x;
    unsigned long long c = 0;
    if (r < g.n_rays) {
        double s[3], w[3];
        exact_ray(g, r, s, w);
        bool ok = true;
        c = count_ray<DEG>(g, s, w, ok, qlo + threadIdx.x, qhi + threadIdx.x);
        if (!ok) atomicOr(g.err, 1);
        if (per_ray) per_ray[r] = (unsigned)c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(total, c);
}

template <int DEG>
spl_status launch_exact(const spl_geometry *g, unsigned long long *total, unsigned *per_ray, cudaStream_t st)
{
    const long long blocks = (g->dev.n_rays + kCountThreads - 1) / kCountThreads;
    k_count_exact<DEG><<<(unsigned)blocks, kCountThreads, 0, st>>>(g->dev, total, per_ray);
    return cuda_check(cudaGetLastError(), "exact count launch");
}

}  // namespace

spl_status count_exact(const spl_geometry *g, int degree, unsigned long long *total, unsigned *per_ray,
                       cudaStream_t st)
{
    if (g->dev.n_rays == 0) return SPL_OK;
    switch (degree) {
    case 0: return launch_exact<0>(g, total, per_ray, st);
    case 1: return launch_exact<1>(g, total, per_ray, st);
    case 2: return launch_exact<2>(g, total, per_ray, st);
    default: return launch_exact<3>(g, total, per_ray, st);
    }
}

}  // namespace spl

extern "C" spl_status spl_count_pairs_per_ray(const spl_geometry *g, int degree, unsigned *per_ray_dev,
                                             unsigned long long *total_dev, void *stream)
{
    spl::clear_error();
    if (!g || (!per_ray_dev && !total_dev)) return spl::fail(SPL_ERR_ARG, "NULL argument");
    if (degree < 0 || degree > 3) return spl::fail(SPL_ERR_ARG, "degree %d not in 0..3", degree);
    unsigned long long *tot = total_dev;
    if (!tot) return spl::fail(SPL_ERR_ARG, "total_dev is NULL");
    return spl::count_exact(g, degree, tot, per_ray_dev, (cudaStream_t)stream);
}
