// spl_host.h -- host-side internals shared by the translation units of
// libspl.so: the geometry object, error reporting and the quadrature rule.
#pragma once

#include <cuda_runtime.h>

#include "spl.h"
#include "spl_march.cuh"

struct spl_geometry {
    spl_geometry_desc desc;       // copy of the description (host pointers cleared)
    spl::DevGeom dev;             // kernel-side view (device pointers)
    spl::ViewPose *views_host;    // host copy of the view poses
    void *dev_block;              // single device allocation: poses/rays + error flag
    int device;
};

namespace spl {

// Record `msg` as the calling thread's last error and return `st`.
spl_status fail(spl_status st, const char *fmt, ...);
// Map a CUDA error to SPL_ERR_CUDA with a message (cudaSuccess -> SPL_OK).
spl_status cuda_check(cudaError_t e, const char *what);
// Clear the thread's last error.
void clear_error();

// Gauss-Legendre rule that integrates degree-3n polynomials exactly
// (m = ceil((3n+1)/2) nodes), computed once per process in FP64.
// (the rule also carries the slab loop bound, see set_iter_cap)
QuadRule quad_rule(int degree);
// Lower the per-slab loop bound for fault-injection tests (1..kSlabIterCap;
// anything else restores the default).  Returns the previous bound.
int set_iter_cap(int cap);
int quad_nodes(int degree);

// Validate a basis descriptor against a geometry (nullable).
spl_status check_basis(const spl_basis_desc *b);

}  // namespace spl
