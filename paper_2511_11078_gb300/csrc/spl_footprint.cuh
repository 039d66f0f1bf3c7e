// spl_footprint.cuh -- the exact footprint Pphi(w, p) of one basis (Eq. 4's
// contribution) on the device: the basis at the origin is a 1x1x1 grid, the
// line {p + t w} is walked with the same march as the projector, and the
// value of the single basis is kept.
#pragma once

#include "spl_march.cuh"

namespace spl {

// the region is the single basis (0, 0, 0); it is the only one put() is
// told is in it, so the strides do not matter
struct PointSink {
    static constexpr bool plane = false;
    static constexpr bool face = false;
    float v;
    int S0 = 0, S1 = 0, S2 = 0;
    unsigned off = 0u;
    struct Box {
        __device__ __forceinline__ bool in0(int d) const { return d == 0; }
        __device__ __forceinline__ bool in1(int a) const { return a == 0; }
        __device__ __forceinline__ bool in2(int b) const { return b == 0; }
        __device__ __forceinline__ bool cube_in(int d0, int a0, int b0, int n) const
        {
            return n == 0 && d0 == 0 && a0 == 0 && b0 == 0;
        }
    } bx;
    __device__ __forceinline__ float wscale() const { return 1.0f; }
    __device__ __forceinline__ void put(unsigned, bool in, float val, int)
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

}  // namespace spl
