// spl_host.h -- host-side internals shared by the translation units of
// libspl.so: the geometry object, error reporting and the quadrature rule.
#pragma once

#include <cuda_runtime.h>

#include "spl.h"
#include "spl_march.cuh"

namespace spl {
struct PlaneGroup;
struct TableSet;
}

struct spl_geometry {
    spl_geometry_desc desc;       // copy of the description (host pointers cleared)
    spl::DevGeom dev;             // kernel-side view (device pointers)
    spl::ViewPose *views_host;    // host copy of the view poses
    void *dev_block;              // single device allocation: poses/rays + error flag
    int device;
    spl::PlaneGroup *plane;       // slice-separable view group (parallel geometries), or NULL
    spl::ViewConst *vconst;       // parallel geometries: per-view constants in view_order order (host)
    spl::TableSet *table;         // footprint tables (SPL_FP_TABLE), built by spl_prepare, or NULL
    double *acc64;                // FP64 accumulator of the scatter adjoint's batches (nx*ny*nz), or NULL
    float *lay[3];                // the scatter adjoint's targets: c in the x-fast [0], y-fast [1] and z-fast [2]
                                  // layouts, four copies each shifted by 0..3 floats (4 * dev.lay_cs floats),
                                  // or NULL (no rays; parallel geometries whose views are all flat)
};

namespace spl {
// The scatter adjoint adds each batch of at most this many views (rays) in
// FP32 atomics and the batches in FP64 (see adjoint_quad).
constexpr int kAdjBatchViews = 48;
constexpr long long kAdjBatchRays = 1LL << 22;
}

namespace spl {

// Plane matrices of a slice-separable view group for one degree (device
// buffers, one allocation).  Row r = (group view g, detector column u) =
// g * nu + u; column = l_q * n_p + l_p (real in-plane indices, p < q).
struct PlanePack {
    int state;                 // 0 not built, 1 built, -1 unavailable (allocation failed)
    void *block;               // allocation of the row/column pointers, weights and scratch
    void *block2;              // allocation of the nnz-sized arrays
    long long nnz;
    long long *row_ptr;        // [rows + 1]
    int *row_col;              // [nnz] columns of each row, in march order
    float *row_val;            // [nnz] G values (1/|w_d| included)
    long long *col_ptr;        // [ncol + 1]
    int *col_row;              // [nnz] rows of each column
    float *col_val;            // [nnz]
    int *lb0;                  // [nv] first b-basis whose support holds detector row v
    float *wz;                 // [nv][degree+1] beta^n(z_v - l_b), l_b = lb0[v] + i
    int *vr;                   // [n_b][2] rows v whose b-window holds basis l_b (inclusive range)
    float *S;                  // [ncol][nv] forward scratch: c resampled along b
    float *T;                  // [ncol][nv] adjoint scratch
    float *yt;                 // [rows][nv] adjoint scratch: y of the group, transposed
};

// Slice-separable view group of a parallel geometry (host object).
struct PlaneGroup {
    int b, p, q;               // separable axis and the in-plane axes (p < q)
    int n_views;               // views in the group: dev.view_order[0 .. n_views)
    long long rows;            // n_views * nu
    long long ncol;            // n_p * n_q
    double z0, dz;             // b index coordinate of detector row v: z0 + v * dz
    PlanePack pack[4];         // per degree
    // The forward runs the plane path on `side` beside the march of the other
    // views (fork and join through the events); NULL when they could not be
    // created (the two then run one after the other).
    cudaStream_t side;
    cudaEvent_t fork, join;
};

// Record `msg` as the calling thread's last error and return `st`.
spl_status fail(spl_status st, const char *fmt, ...);
// Map a CUDA error to SPL_ERR_CUDA with a message (cudaSuccess -> SPL_OK).
spl_status cuda_check(cudaError_t e, const char *what);
// Clear the thread's last error.
void clear_error();
// Number of SMs of the current device (queried once per device).
int sm_count();
// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, once per kernel and device (thread-safe).
spl_status smem_attr_once(const void *func, int bytes, const char *what);

// Gauss-Legendre rule that integrates degree-3n polynomials exactly
// (m = ceil((3n+1)/2) nodes), computed once per process in FP64.
// (the rule also carries the event-loop bound, see set_iter_cap)
QuadRule quad_rule(int degree);
// Lower the event-loop bound for fault-injection tests (1..kIterCap;
// anything else restores the default).  Returns the previous bound.
int set_iter_cap(int cap);
int quad_nodes(int degree);

// Exact pair count (count.cu): adds to *total, per ray into per_ray (nullable).
spl_status count_exact(const spl_geometry *g, int degree, unsigned long long *total, unsigned *per_ray,
                       cudaStream_t st);

// Validate a basis descriptor against a geometry (nullable).
spl_status check_basis(const spl_basis_desc *b);

// Plane-matrix path of slice-separable views (plane.cu).  plane_ready
// builds the degree's pack on first use; false when the geometry has no
// group or the pack is unavailable.
bool plane_ready(spl_geometry *g, int degree, cudaStream_t st, spl_status *err);
// State of the degree's pack without building it: 0 not built, 1 built, -1
// unavailable (allocation failed, or no separable group).
int plane_state(const spl_geometry *g, int degree);
spl_status plane_forward(const spl_geometry *g, int degree, int kahan, const float *c, float *y, cudaStream_t st);
// writes every coefficient (the other views' scatter adds after it)
spl_status plane_adjoint(const spl_geometry *g, int degree, const float *y, float *c, cudaStream_t st);
// The adjoint's two stages: T (the column gather of y) into the pack's
// scratch, then c += the b-resampled T (the forward of the same geometry
// must not run in between).
spl_status plane_adjoint_t(const spl_geometry *g, int degree, const float *y, cudaStream_t st);
spl_status plane_adjoint_add(const spl_geometry *g, int degree, float *c, cudaStream_t st);
void plane_free(PlaneGroup *pg);

// Footprint tables of the views of a parallel geometry (table.cu): built
// by table_build (spl_prepare); the projector returns SPL_ERR_STATE when
// they are missing.
spl_status table_build(spl_geometry *g, int degree, cudaStream_t st);
spl_status table_forward(const spl_geometry *g, const spl_basis_desc *b, const float *c, float *y, cudaStream_t st);
spl_status table_adjoint(const spl_geometry *g, const spl_basis_desc *b, const float *y, float *c, cudaStream_t st);
void table_free(TableSet *ts);

}  // namespace spl
