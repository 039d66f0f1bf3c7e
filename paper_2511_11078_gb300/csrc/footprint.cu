// footprint.cu -- batched footprint Pphi(w, p) (Eq. 4's contribution) and
// the MLP input features.
//
// Exact mode: the basis at the origin is a 1x1x1 grid; the ray {p + t w} is
// set up and walked with the same cell march as the projector, and the
// value of the single basis is kept.  MLP mode: f_theta on the canonical features,
// times the exact support indicator (the same pair test as the projector).
#include "spl_host.h"
#include "spl_mlp.cuh"

namespace spl {

// the region is the single basis (0, 0, 0); it is the only one put() is
// told is in it, so the strides do not matter
struct PointSink {
    static constexpr bool plane = false;
    float v;
    int S0 = 0, S1 = 0, S2 = 0;
    unsigned off = 0u;
    struct Box {
        __device__ __forceinline__ bool in0(int d) const { return d == 0; }
        __device__ __forceinline__ bool in1(int a) const { return a == 0; }
        __device__ __forceinline__ bool in2(int b) const { return b == 0; }
    } bx;
    __device__ __forceinline__ void put(unsigned, bool in, float val)
    {
        if (in) v = val;
    }
    __device__ __forceinline__ void piece() {}
    __device__ __forceinline__ bool relevant(int d0, int d1, int a0, int a1, int b0, int b1) const
    {
        return d0 <= 0 && d1 >= 0 && a0 <= 0 && a1 >= 0 && b0 <= 0 && b1 >= 0;
    }
    __device__ __forceinline__ void flush(int ld, int la, int lb, float val)
    {
        if (ld == 0 && la == 0 && lb == 0) v = val;
    }
    __device__ __forceinline__ void cell_end() {}
};

__device__ __forceinline__ GridBox unit_box()
{
    GridBox gb;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        gb.n[e] = 1;
        gb.org[e] = 0.0;
        gb.stride[e] = 1;
    }
    return gb;
}

template <int N>
__device__ __forceinline__ float footprint_exact(const double (&w)[3], const double (&p)[3], const QuadRule &qr)
{
    RaySetup rs;
    if (!ray_setup<N>(unit_box(), p, w, rs)) return 0.0f;
    PointSink sk;
    sk.v = 0.0f;
    march<N>(rs, rs.c0, rs.c1, qr, sk);
    return sk.v * rs.inv_wd;
}

template <int N>
__global__ void k_footprint_quad(long long count, const float *__restrict__ omega, const float *__restrict__ p,
                                 float *__restrict__ out, QuadRule qr)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double w[3], q[3];
    double nrm = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        w[e] = omega[3 * i + e];
        q[e] = p[3 * i + e];
        nrm += w[e] * w[e];
    }
    nrm = sqrt(nrm);
    if (!(nrm > 0.0)) {
        out[i] = 0.0f;
        return;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) w[e] /= nrm;
    out[i] = footprint_exact<N>(w, q, qr);
}

__global__ void k_features(int degree, long long count, const float *__restrict__ omega, const float *__restrict__ p,
                           float *__restrict__ feat)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double w[3], q[3], f[5];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        w[e] = omega[3 * i + e];
        q[e] = p[3 * i + e];
    }
    canonical_features(degree, w, q, f);
#pragma unroll
    for (int e = 0; e < 5; ++e) feat[5 * i + e] = (float)f[e];
}

// Algorithm 1's training distribution from caller-drawn random numbers:
// w = n / |n| (n standard normal: uniform on the sphere), p uniform in the
// disc of radius sqrt(3) W of H_w: p = r (cos a u + sin a v) with
// r = sqrt(3) W sqrt(u1), a = 2 pi u2 and (u, v) an orthonormal pair
// perpendicular to w.
__global__ void k_samples(int degree, long long count, const float *__restrict__ normals,
                          const float *__restrict__ uniforms, float *__restrict__ omega, float *__restrict__ p)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double w[3];
    double nrm = 0.0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        w[e] = normals[3 * i + e];
        nrm += w[e] * w[e];
    }
    nrm = sqrt(nrm);
    if (!(nrm > 0.0)) {
        w[0] = 0.0;
        w[1] = 0.0;
        w[2] = 1.0;
        nrm = 1.0;
    } else {
#pragma unroll
        for (int e = 0; e < 3; ++e) w[e] /= nrm;
    }
    // u = normalize(ref x w) with ref = e3 unless w is close to e3
    const double ref[3] = {fabs(w[2]) < 0.9 ? 0.0 : 1.0, 0.0, fabs(w[2]) < 0.9 ? 1.0 : 0.0};
    double u[3] = {ref[1] * w[2] - ref[2] * w[1], ref[2] * w[0] - ref[0] * w[2], ref[0] * w[1] - ref[1] * w[0]};
    const double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
    for (int e = 0; e < 3; ++e) u[e] /= un;
    const double v[3] = {w[1] * u[2] - w[2] * u[1], w[2] * u[0] - w[0] * u[2], w[0] * u[1] - w[1] * u[0]};
    const double W = 0.5 * (degree + 1);
    const double r = sqrt(3.0) * W * sqrt((double)uniforms[2 * i]);
    const double a = 6.283185307179586 * (double)uniforms[2 * i + 1];
    const double ca = cos(a), sa = sin(a);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        omega[3 * i + e] = (float)w[e];
        p[3 * i + e] = (float)(r * (ca * u[e] + sa * v[e]));
    }
}

}  // namespace spl

using namespace spl;

template <int N>
static spl_status footprint_quad(long long count, const float *w, const float *p, float *out, cudaStream_t st)
{
    const long long blocks = (count + 127) / 128;
    k_footprint_quad<N><<<(unsigned)blocks, 128, 0, st>>>(count, w, p, out, quad_rule(N));
    return cuda_check(cudaGetLastError(), "footprint launch");
}

extern "C" spl_status spl_footprint(const spl_basis_desc *b, long long count, const float *omega_dev,
                                    const float *p_dev, float *out_dev, void *stream)
{
    clear_error();
    spl_status s = check_basis(b);
    if (s != SPL_OK) return s;
    if (count < 0 || count > (1LL << 40)) return fail(SPL_ERR_ARG, "bad count %lld", count);
    if (count == 0) return SPL_OK;
    if (!omega_dev || !p_dev || !out_dev) return fail(SPL_ERR_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->mode == SPL_FP_MLP) {
        if (spl_mlp_degree(b->mlp) != b->degree) return fail(SPL_ERR_ARG, "MLP degree does not match basis degree");
        return spl::footprint_mlp(b, count, omega_dev, p_dev, out_dev, st);
    }
    switch (b->degree) {
    case 0: return footprint_quad<0>(count, omega_dev, p_dev, out_dev, st);
    case 1: return footprint_quad<1>(count, omega_dev, p_dev, out_dev, st);
    case 2: return footprint_quad<2>(count, omega_dev, p_dev, out_dev, st);
    default: return footprint_quad<3>(count, omega_dev, p_dev, out_dev, st);
    }
}

extern "C" spl_status spl_features(int degree, long long count, const float *omega_dev, const float *p_dev,
                                   float *feat_dev, void *stream)
{
    clear_error();
    if (degree < 0 || degree > 3) return fail(SPL_ERR_ARG, "degree %d not in 0..3", degree);
    if (count < 0) return fail(SPL_ERR_ARG, "bad count");
    if (count == 0) return SPL_OK;
    if (!omega_dev || !p_dev || !feat_dev) return fail(SPL_ERR_ARG, "NULL array");
    const long long blocks = (count + 127) / 128;
    k_features<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(degree, count, omega_dev, p_dev, feat_dev);
    return cuda_check(cudaGetLastError(), "features launch");
}

extern "C" spl_status spl_footprint_samples(int degree, long long count, const float *normals_dev,
                                            const float *uniforms_dev, float *omega_dev, float *p_dev, void *stream)
{
    clear_error();
    if (degree < 0 || degree > 3) return fail(SPL_ERR_ARG, "degree %d not in 0..3", degree);
    if (count < 0) return fail(SPL_ERR_ARG, "bad count");
    if (count == 0) return SPL_OK;
    if (!normals_dev || !uniforms_dev || !omega_dev || !p_dev) return fail(SPL_ERR_ARG, "NULL array");
    const long long blocks = (count + 127) / 128;
    k_samples<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(degree, count, normals_dev, uniforms_dev, omega_dev,
                                                                  p_dev);
    return cuda_check(cudaGetLastError(), "samples launch");
}
