// spl_mlp.cuh -- learned footprint f_theta (Sec. 2.2, Algorithm 1): shared
// declarations and the canonical input features.
#pragma once

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
// (Gw1, Gw2, Gw3, <Gp,u>/(sqrt3 W), <Gp,v>/(sqrt3 W)).  FP64.
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
    const double sc = 1.0 / (sqrt(3.0) * W);
    f[0] = w[0];
    f[1] = w[1];
    f[2] = w[2];
    f[3] = (p[0] * u[0] + p[1] * u[1] + p[2] * u[2]) * sc;
    f[4] = (p[0] * v[0] + p[1] * v[1] + p[2] * v[2]) * sc;
}

spl_status forward_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st);
spl_status adjoint_mlp(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st);
spl_status footprint_mlp(const spl_basis_desc *b, long long count, const float *w, const float *p, float *out,
                         cudaStream_t st);

}  // namespace spl
