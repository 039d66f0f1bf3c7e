// footprint.cu -- batched footprint Pphi(w, p) (Eq. 4's contribution) and
// the MLP input features.
//
// Exact mode: the basis at the origin is a 1x1x1 grid; the ray {p + t w} is
// set up and walked with the same cell march as the projector, and the
// value of the single basis is kept.  MLP mode: f_theta on the canonical features,
// times the exact support indicator (the same pair test as the projector).
#include "spl_footprint.cuh"
#include "spl_host.h"
#include "spl_mlp.cuh"

namespace spl {

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

extern "C" spl_status spl_frame(long long count, const double *omega, double *u, double *v)
{
    clear_error();
    if (count < 0) return fail(SPL_ERR_ARG, "bad count");
    if (count == 0) return SPL_OK;
    if (!omega || !u || !v) return fail(SPL_ERR_ARG, "NULL array");
    for (long long i = 0; i < count; ++i) {
        double w[3];
        double nrm = 0.0;
        for (int e = 0; e < 3; ++e) {
            w[e] = omega[3 * i + e];
            nrm += w[e] * w[e];
        }
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) return fail(SPL_ERR_NONFINITE, "direction %lld is zero or not finite", i);
        for (int e = 0; e < 3; ++e) w[e] /= nrm;
        double uu[3], vv[3];
        canonical_frame(w, uu, vv);
        for (int e = 0; e < 3; ++e) {
            u[3 * i + e] = uu[e];
            v[3 * i + e] = vv[e];
        }
    }
    return SPL_OK;
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
