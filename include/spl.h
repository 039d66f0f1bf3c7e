/*
 * spl.h -- C ABI of libspl.so: the x-ray transform of a volume expanded in
 * tensor-product B-splines (SplineSplat, arXiv 2511.11078), its adjoint, the
 * basis footprint (exact or learned), the learned-footprint MLP and the FP64
 * reductions of least-squares reconstruction, all as hand-written CUDA
 * kernels for sm_103a (GB300).
 *
 * Model (paper Sec. 1.2, Eq. 1-4):
 *   f(x) = sum_{k in grid} c_k beta^n(x1-X1(k)) beta^n(x2-X2(k)) beta^n(x3-X3(k))
 *   with X(k) = origin + k (unit lattice, Sec. 2.1) and beta^n the centred
 *   B-spline of degree n (Sec. 2.2 uses n = 2; any n in 0..3 here).
 *   A ray is the line {s + t w}, |w| = 1 (Eq. 1).  Its value is the line
 *   integral of f (Eq. 2) = sum_k c_k Pphi(w, s - X(k)) (Eq. 4), where the
 *   footprint Pphi(w, p) = int prod_d beta^n(p_d + t w_d) dt is the
 *   "contribution" of basis k.  A (ray, basis) pair counts when the line
 *   meets the open support cube of the basis in a segment of positive length.
 *
 * Common conventions
 *   - Coefficients: float32, C-order c[z][y][x] (x fastest), nx*ny*nz values.
 *   - Projections: float32, y[view][v][u] for view geometries, y[ray] for
 *     explicit rays.
 *   - "_dev" pointers are device pointers owned by the caller; the library
 *     never frees them and never keeps them after the call returns.
 *   - Every compute call is asynchronous on the CUDA stream `stream`
 *     (a cudaStream_t, NULL for the legacy default stream).  Argument errors
 *     are detected before any launch and returned synchronously; the call
 *     then launches nothing.
 *   - spl_forward, spl_adjoint, spl_footprint, spl_dot_f64 and the CG updates
 *     allocate no memory.  Objects (geometry, MLP) own the device memory they
 *     allocate at creation (and, for a geometry, in spl_prepare) and free it
 *     on destroy.  A basis whose structures a geometry has not built
 *     (spl_prepare) is refused by spl_forward / spl_adjoint with
 *     SPL_ERR_STATE.
 *   - Errors are returned as spl_status values; the library never aborts.
 *     spl_last_error() gives a message for the last failing call of the
 *     calling thread.
 *   - Kernels never spin on a condition another agent sets; every loop has a
 *     fixed bound.  A kernel that reaches a bound sets the error flag of the
 *     geometry it ran on; spl_geometry_status() reads and clears it.  The
 *     tensor-core kernels wait for their MMAs with a bounded poll; a wait
 *     that gives up sets the error flag of the geometry (projector) or of
 *     the network (spl_footprint, spl_mlp_eval, training), reported as
 *     SPL_ERR_TIMEOUT by spl_geometry_status() / spl_mlp_status().
 */
#ifndef SPL_H
#define SPL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPL_OK = 0,
    SPL_ERR_ARG = 1,         /* null pointer, bad size, bad degree or mode      */
    SPL_ERR_NONFINITE = 2,   /* non-finite or zero-length direction or position */
    SPL_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
    SPL_ERR_STEPCAP = 4,     /* a kernel reached one of its loop bounds         */
    SPL_ERR_OOM = 5,         /* device allocation failed (object creation only) */
    SPL_ERR_STATE = 6,       /* object in the wrong state for this call         */
    SPL_ERR_UNSUPPORTED = 7, /* size or option outside what the kernels handle  */
    SPL_ERR_TIMEOUT = 8      /* a bounded tensor-core completion wait gave up   */
} spl_status;

/* geometry kinds (Eq. 1 lines) */
enum { SPL_RAYS = 0, SPL_PARALLEL = 1, SPL_CONE = 2 };
/* footprint evaluators: exact quadrature, or the learned f_theta (Sec. 2.2);
 * SPL_FP_DIRECT: exact too, but spl_forward integrates f itself along the
 * ray (the Gauss nodes of the same pieces, a window of coefficients instead
 * of footprint accumulators) on rays with three nonzero direction
 * components; everything else is as SPL_FP_QUAD (same matrix). */
enum { SPL_FP_QUAD = 0, SPL_FP_MLP = 1, SPL_FP_DIRECT = 2, SPL_FP_TABLE = 3 };
/* SPL_FP_TABLE (parallel-beam geometries only): the splat form, an
 * approximation.  Each view's footprint, one 2-D function on H_w, is
 * tabulated exactly on a grid of step h = 1/32 in the frame
 * e1 = (det_u - (det_u.w) w)/|...|, e2 = w x e1, at the nodes
 * (i - M) h e1 + (j - M) h e2, i, j = 0..2M, M = ceil(sqrt(3)(n+1)/(2h)) + 1,
 * and a pair's footprint is the bilinear interpolation of the table at the
 * pair's offset (second-order accurate in h), over the exact pair set.  The
 * tables (4 (2M+1)^2 bytes per view, 198 KB for cubic) are built by
 * spl_prepare (device allocation and kernels, then a synchronisation).
 * Forward and adjoint use the same table values; other geometry kinds
 * return SPL_ERR_UNSUPPORTED.  spl_footprint with this mode,
 * or with SPL_FP_DIRECT, evaluates the exact footprint. */
/* adjoint forms for view geometries: SPL_ADJ_AUTO picks the faster one on
 * this GPU (the scatter form); SPL_ADJ_GATHER walks coefficient bricks and
 * accumulates in shared memory (no global atomics); SPL_ADJ_SCATTER walks
 * rays like spl_forward and adds with float atomics to global memory.  Both
 * visit the same pairs with the same footprint values; both add in an
 * order that varies between runs (float atomics in shared or global
 * memory), so results agree to rounding, not bit for bit. */
enum { SPL_ADJ_AUTO = 0, SPL_ADJ_GATHER = 1, SPL_ADJ_SCATTER = 2 };
/* slice-separable parallel views (see spl_prepare): SPL_SEP_AUTO uses the
 * plane-matrix path for them, SPL_SEP_OFF walks them like any other view */
enum { SPL_SEP_AUTO = 0, SPL_SEP_OFF = 1 };

typedef struct spl_geometry spl_geometry; /* opaque, library-owned */
typedef struct spl_mlp spl_mlp;           /* opaque, library-owned */

/* Description of a set of lines (Eq. 1) and of the coefficient grid.
 *   kind SPL_RAYS:     n_rays lines; ray_omega [n_rays][3] (any nonzero
 *                      length, normalised by the library), ray_s [n_rays][3].
 *   kind SPL_PARALLEL: n_views views of nu x nv pixels; view_src [n_views][3]
 *                      is the ray direction of the view.
 *   kind SPL_CONE:     view_src [n_views][3] is the source position.
 *   For both view kinds pixel (iu, iv) of view k has centre
 *     q = det_center[k] + (iu - (nu-1)/2) det_u[k] + (iv - (nv-1)/2) det_v[k]
 *   (det_u and det_v carry the pixel pitch); the ray is q + t*dir (parallel)
 *   or the line through the source and q (cone); ray index
 *   r = (k*nv + iv)*nu + iu.  All arrays are host FP64, read during the call
 *   and copied to the device; the caller keeps ownership.
 *   Grid: coefficient (i, j, l) sits at origin + (i, j, l), lattice step 1
 *   (Sec. 2.1 places the bases on the unit lattice).  A grid of step h is
 *   the same transform in units of h: divide every position (origin,
 *   sources, detector centres and axes, ray points) by h and multiply the
 *   forward projection (and the adjoint) by h. */
typedef struct {
    int kind;
    int nx, ny, nz;
    double origin[3];
    long long n_rays;
    const double *ray_omega;
    const double *ray_s;
    int n_views;
    const double *view_src;
    const double *det_center;
    const double *det_u;
    const double *det_v;
    int nu, nv;
} spl_geometry_desc;

/* Basis and footprint choice.
 *   degree: n in 0..3 (B-spline degree of the tensor-product basis).
 *   mode:   SPL_FP_QUAD (exact piecewise Gauss-Legendre footprint),
 *           SPL_FP_DIRECT (the same operator; forward as the direct line
 *           integral of f), SPL_FP_TABLE (tabulated footprints, parallel
 *           beams) or SPL_FP_MLP (learned footprint f_theta, Algorithm 2's
 *           f_theta*);
 *           SPL_FP_MLP needs `mlp` built for the same degree.
 *   kahan:  nonzero = compensated (Kahan) FP32 sum of the slab partials along
 *           each ray; zero = plain FP32 sum.
 *   adjoint: form of spl_adjoint on view geometries (see SPL_ADJ_*).
 *   separable: SPL_SEP_AUTO (0) or SPL_SEP_OFF: whether the slice-separable
 *           views of a parallel geometry take the plane-matrix path
 *           (exact quadrature only). */
typedef struct {
    int degree;
    int mode;
    const spl_mlp *mlp;
    int kahan;
    int adjoint;   /* SPL_ADJ_AUTO (0), SPL_ADJ_GATHER or SPL_ADJ_SCATTER; view geometries only */
    int separable; /* SPL_SEP_AUTO (0) or SPL_SEP_OFF */
} spl_basis_desc;

/* ---------------------------------------------------------------- geometry */

/* Build a device-resident geometry (Eq. 1) from `desc`.  Validates every
 * direction and position (finite, nonzero direction) and the grid
 * (1 <= n <= 2048 per axis, nx*ny*nz < 2^31).  Allocates device memory owned
 * by the returned object; a parallel geometry with slice-separable views also
 * owns a CUDA stream and two events on which spl_forward / spl_adjoint run
 * the plane path beside the march of the other views (the caller's stream
 * waits for it, so each call stays one ordered operation on that stream).
 * Scratch of the scatter adjoint, allocated here: the coefficient array in
 * three layouts (x, y and z fast) of four shifted copies each (about
 * 48 nx ny nz bytes; not for a parallel geometry whose views are all in the
 * flat class) and, for more than 48 views or 2^22 explicit rays, an FP64
 * accumulator (8 nx ny nz bytes).
 * Uses the current CUDA device.
 * Errors: SPL_ERR_ARG, SPL_ERR_NONFINITE, SPL_ERR_UNSUPPORTED, SPL_ERR_OOM,
 * SPL_ERR_CUDA; *out is NULL on error. */
spl_status spl_make_geometry(const spl_geometry_desc *desc, spl_geometry **out);

/* Free a geometry (NULL is ignored).  No call using it may be in flight. */
void spl_destroy_geometry(spl_geometry *g);

/* Number of rays (= length of y) and of coefficients (= length of c). */
long long spl_geometry_rays(const spl_geometry *g);
long long spl_geometry_coeffs(const spl_geometry *g);

/* Synchronise `stream`, then read and clear the geometry's device error flag.
 * Returns SPL_ERR_TIMEOUT if a tensor-core wait of the learned-footprint
 * projector gave up, else SPL_ERR_STEPCAP if a kernel that ran on `g`
 * reached a loop bound since the last call, SPL_ERR_CUDA on a CUDA error,
 * else SPL_OK. */
spl_status spl_geometry_status(const spl_geometry *g, void *stream);

/* Slice-separable views.  A parallel view is slice-separable along axis b
 * when its direction has a zero b component and its detector rows run
 * along b: det_u has no b component and det_v has only one.  The rays of
 * such a view are flat, so a footprint factors exactly,
 *   Pphi(w, s - l) = G(u; l_p, l_q) * beta^n(z_v - l_b),
 * with G the footprint of the 2-D tensor B-spline in the plane of the other
 * two axes (p, q) and z_v the b coordinate of detector row v.  All rows of a
 * detector column then share one plane path, and
 *   y(u, v) = sum_(l_p, l_q) G(u; l_p, l_q) * S(l_p, l_q; v),
 *   S(l_p, l_q; v) = sum_(l_b) beta^n(z_v - l_b) c_l.
 * The views of one separable group (the largest set that shares b, the b
 * coordinate of the detector centre and the b step of det_v) take this
 * path: the plane matrix G of the group (one row per view and detector
 * column, one column per (l_p, l_q); its values come from the same flat cell
 * march as every other ray) is built once per degree, with its transpose;
 * a forward then resamples c along b into S and gathers the rows of G;
 * an adjoint gathers the columns of G and resamples back along b, with no
 * atomics.
 * spl_prepare builds what spl_forward / spl_adjoint need for `basis` on
 * this geometry, which they never allocate themselves: the plane matrices
 * for basis->degree (exact footprint, SPL_SEP_AUTO, geometries with a
 * separable group), or the footprint tables of SPL_FP_TABLE (see there).
 * One-time device allocation and kernels on `stream`, then a
 * synchronisation; later calls for the same degree return at once.  Until
 * it has run, spl_forward / spl_adjoint refuse such a basis with
 * SPL_ERR_STATE.  Geometries without separable views,
 * basis->separable == SPL_SEP_OFF and the MLP footprint need nothing.  The
 * plane buffers include the scratch of S and of its adjoint, so calls on
 * one geometry must not overlap on the GPU.
 * Errors: SPL_ERR_ARG; SPL_ERR_OOM (plane matrices: the path stays off for
 * this geometry and degree, and spl_forward / spl_adjoint then walk those
 * views like the others and succeed; tables: SPL_FP_TABLE stays
 * unavailable); SPL_ERR_UNSUPPORTED (SPL_FP_TABLE on a cone or ray
 * geometry); SPL_ERR_CUDA. */
spl_status spl_prepare(spl_geometry *g, const spl_basis_desc *basis, void *stream);

/* ---------------------------------------------------------------- operators */

/* Forward projection y = A c (Algorithm 2; Eq. 4 summed over all pairs).
 * One GPU thread per ray marches the unit cells of the ray's dominant axis
 * (Definition 2.1); an (n+1)^3 window holds the bases whose support contains
 * the current point (Algorithm 3's neighbourhood, de-duplicated by
 * construction), and each basis the ray crosses adds c_k * Pphi(w, s - X(k))
 * once.  Slice-separable views of a parallel geometry go through the plane
 * matrices instead (see spl_prepare), with the same footprint values.
 *   Cone views: every ray is walked with the general (three-factor) form
 *   of the march, so a ray's values do not depend on its direction class.
 *   c_dev: [nz][ny][nx] float32 (read only);  y_dev: n_rays float32,
 *   overwritten.  Errors: SPL_ERR_ARG (null pointer, degree, mode, missing or
 *   mismatched MLP), SPL_ERR_STATE (the basis needs spl_prepare first),
 *   SPL_ERR_CUDA (launch failure). */
spl_status spl_forward(const spl_geometry *g, const spl_basis_desc *basis, const float *c_dev, float *y_dev,
                       void *stream);

/* Adjoint (back-projection) c = A^T y: the transpose of the matrix of Eq. 6,
 * matched exactly to spl_forward (Sec. 2.3): it visits the same
 * (ray, basis) pairs and evaluates bit-identical footprint values.  View
 * geometries use the form chosen by basis->adjoint (SPL_ADJ_*): a
 * ray-driven scatter with float atomics (the default) or a gather over
 * coefficient bricks that loops over views and the detector window of the
 * brick (no global atomics); explicit rays always scatter.  The scatter
 * reduces each ray into the geometry's layout of c whose contiguous axis
 * is the ray's smallest direction component and folds the layouts into
 * c_dev (so two calls on one geometry must not overlap on the GPU).  Slice-separable
 * views of a parallel geometry are gathered through the transposed plane
 * matrix (no atomics; see spl_prepare) and the other views added to them.
 *   y_dev: n_rays float32 (read only);  c_dev: [nz][ny][nx] float32,
 *   overwritten.  Errors as spl_forward. */
spl_status spl_adjoint(const spl_geometry *g, const spl_basis_desc *basis, const float *y_dev, float *c_dev,
                       void *stream);

/* Work of one forward projection, added to count_dev (uint64 [3], device):
 * count_dev[0] += number of contributions of Eq. 4: (ray, basis) pairs whose
 * line meets the open support cube of the basis in a segment of positive
 * length, decided exactly as spl_count_pairs_per_ray does;
 * count_dev[1] += pieces the march integrates with the full Gauss-Legendre
 * rule of ceil((3n+1)/2) nodes (rays with three nonzero direction
 * components, and every cone ray); count_dev[2] += pieces of parallel and
 * explicit rays with a zero component (n+1 nodes each: the third factor is
 * constant along the ray). */
spl_status spl_count_pairs(const spl_geometry *g, int degree, unsigned long long *count_dev, void *stream);

/* The contributions of Eq. 4 ray by ray: per_ray_dev[r] (uint32, n_rays,
 * nullable) = the number of bases k of the grid whose open support cube
 * [k - W, k + W]^3 (W = (n+1)/2) the line of ray r meets in a segment of
 * positive length, and *total_dev (uint64, device) += their sum.  The
 * decision is made in FP64 with the plain definition's operations, each
 * rounded separately (no fused multiply-add): the ray is rebuilt from the
 * caller's arrays as given (pixel centre (det_center + a det_u) + b det_v,
 * direction over sqrt((d0 d0 + d1 d1) + d2 d2)); along each axis e with
 * w_e != 0, p = s_e - (origin_e + k_e) and the line is inside the support
 * slab for t between (-W - p)/w_e and (W - p)/w_e; along an axis with
 * w_e = 0, k_e is admitted when the truncated-power B-spline sum
 * (1/n!) sum_j (-1)^j C(n+1,j) (W - |p| - j)_+^n is positive (degree 0:
 * -1/2 <= p < 1/2); a pair counts when the largest lower end is below the
 * smallest upper end.  Errors: SPL_ERR_ARG; the geometry's error flag
 * (SPL_ERR_STEPCAP) if a ray's interval queue overflowed (not expected). */
spl_status spl_count_pairs_per_ray(const spl_geometry *g, int degree, unsigned *per_ray_dev,
                                   unsigned long long *total_dev, void *stream);

/* Footprint Pphi(w, p) (Eq. 4's contribution) of the basis at the origin for
 * `count` (direction, offset) pairs.
 *   omega_dev [count][3] float32 unit directions, p_dev [count][3] float32
 *   offsets (only the component in H_w matters), out_dev [count] float32.
 *   SPL_FP_QUAD: exact knot-split Gauss-Legendre; SPL_FP_MLP: f_theta on the
 *   canonical features, multiplied by the exact support indicator. */
spl_status spl_footprint(const spl_basis_desc *basis, long long count, const float *omega_dev, const float *p_dev,
                         float *out_dev, void *stream);

/* The frame of H_w in which spl_features measures offsets, for `count`
 * directions (host arrays, FP64 [count][3]; any nonzero length, normalised
 * here).  Algorithm 2 fixes only u perpendicular to w and v = u x w; the
 * library's frame is continuous over the chamber 0 <= w1 <= w2 <= w3 of
 * the direction's signed permutation G (phi is invariant under G): there
 * u_c = normalize(e1 x Gw), v_c = u_c x Gw, and the outputs are
 * u = G^T u_c, v = G^T v_c (orthonormal, perpendicular to w,
 * v = det(G) u x w).  spl_features' last two values are <p, u> sqrt(3)/W
 * and <p, v> sqrt(3)/W.  Synchronous host call, no device work.
 * Errors: SPL_ERR_ARG, SPL_ERR_NONFINITE (zero or non-finite direction). */
spl_status spl_frame(long long count, const double *omega, double *u, double *v);

/* MLP input features of (w, p) (float32 [count][5]): the signed permutation
 * G that maps w into the chamber 0 <= w1 <= w2 <= w3 (phi is invariant under
 * it), the frame u = normalize(e1 x Gw), v = u x Gw (Algorithm 2 fixes only
 * u perpendicular to w and v = u x w), and
 * (Gw1, Gw2, Gw3, <Gp,u> sqrt(3)/W, <Gp,v> sqrt(3)/W), W = (n+1)/2 (the
 * sampling disc of radius sqrt(3) W maps to radius 3). */
spl_status spl_features(int degree, long long count, const float *omega_dev, const float *p_dev, float *feat_dev,
                        void *stream);

/* ---------------------------------------------------------------- learned footprint (Sec. 2.2, Algorithm 1) */

/* Training samples of Algorithm 1 from caller-drawn random numbers (the
 * caller owns the generator): normals_dev [count][3] standard normal,
 * uniforms_dev [count][2] in [0, 1).  Writes unit directions
 * w = n/|n| (uniform on the sphere) to omega_dev [count][3] and offsets p,
 * uniform in the disc of radius sqrt(3) W = sqrt(3)(n+1)/2 of H_w, to
 * p_dev [count][3] (the disc contains the whole footprint support). */
spl_status spl_footprint_samples(int degree, long long count, const float *normals_dev, const float *uniforms_dev,
                                 float *omega_dev, float *p_dev, void *stream);



/* The network is fixed: 5 -> 64 -> 64 -> 64 -> 1, SiLU after the three
 * hidden layers.  Parameters (float32 master copy) are laid out per layer as
 * W [out][in] row-major followed by b [out]; SPL_MLP_PARAMS values in all.
 * Evaluation precision: BF16 weights (rounded from the master copy), BF16
 * hidden activations into the two 64x64 tensor-core layers, FP32
 * accumulation, FP32 first and last layers. */
#define SPL_MLP_PARAMS 8769

/* Create an MLP for B-splines of `degree`, parameters initialised with a
 * seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) draw; allocates device
 * memory (weights, Adam state, and training scratch for batches of up to
 * `max_batch` samples).  Errors: SPL_ERR_ARG, SPL_ERR_OOM, SPL_ERR_CUDA. */
spl_status spl_mlp_create(int degree, int max_batch, unsigned long long seed, spl_mlp **out);
void spl_mlp_destroy(spl_mlp *m);
int spl_mlp_degree(const spl_mlp *m);

/* Copy SPL_MLP_PARAMS float32 master parameters from / to the host
 * (synchronous).  Setting also refreshes the BF16 copies and resets Adam. */
spl_status spl_mlp_set_params(spl_mlp *m, const float *host_params);
spl_status spl_mlp_get_params(const spl_mlp *m, float *host_params);

/* f_theta on `count` feature rows (float32 [count][5]) -> out_dev [count],
 * on the tcgen05 tensor cores (128-row tiles, BF16 operands, FP32
 * accumulation in tensor memory; layer 1 and the biases at FP32 accuracy).
 * A tensor-core completion wait that exceeds its bound (not expected)
 * leaves NaN in the rows of the affected tile and sets the network's error
 * flag (spl_mlp_status). */
spl_status spl_mlp_eval(const spl_mlp *m, long long count, const float *feat_dev, float *out_dev, void *stream);

/* Synchronise `stream`, then read and clear the network's device error
 * flag: SPL_ERR_TIMEOUT if a tensor-core wait of spl_footprint
 * (SPL_FP_MLP), spl_mlp_eval, spl_mlp_grad or spl_mlp_train_step on this
 * network gave up since the last call, else SPL_OK (SPL_ERR_CUDA on a CUDA
 * error). */
spl_status spl_mlp_status(const spl_mlp *m, void *stream);

/* Checkpoint of the training state (Algorithm 1), a little-endian binary
 * file: the 8 bytes "SPLMLP2\0"; int32 version (2), degree, parameter count
 * (SPL_MLP_PARAMS), input width (5), hidden width (64), hidden layers (3),
 * dtype (0 = float32), Adam step count; uint64 initialisation seed; then
 * the float32 master parameters, Adam first moments and Adam second
 * moments (SPL_MLP_PARAMS values each).  spl_mlp_load restores all of it
 * (and refreshes the BF16 copies), so training resumes exactly where the
 * saved network stopped.  Both synchronise the device.  spl_mlp_load
 * refuses a file of another degree or shape (SPL_ERR_ARG) and non-finite
 * values (SPL_ERR_NONFINITE); I/O failures return SPL_ERR_ARG with the
 * reason in spl_last_error(). */
spl_status spl_mlp_save(const spl_mlp *m, const char *path);
spl_status spl_mlp_load(spl_mlp *m, const char *path);

/* Gradient of L = (1/B) sum_b (f_theta(x_b) - y_b)^2 (Algorithm 1's loss)
 * with respect to the master parameters, float32 [SPL_MLP_PARAMS] into
 * grad_dev; the loss into loss_dev (float32 [1]).  B <= max_batch. */
spl_status spl_mlp_grad(spl_mlp *m, int batch, const float *feat_dev, const float *target_dev, float *grad_dev,
                        float *loss_dev, void *stream);

/* One Adam step (Algorithm 1's update) on a batch: gradient as
 * spl_mlp_grad, then Adam with learning rate `lr` (beta1 0.9, beta2 0.999,
 * eps 1e-8) on the FP32 master weights, then the BF16 copies refresh.
 * loss_dev (nullable) receives the batch loss. */
spl_status spl_mlp_train_step(spl_mlp *m, int batch, const float *feat_dev, const float *target_dev, float lr,
                              float *loss_dev, void *stream);

/* ---------------------------------------------------------------- FP64 reductions (Eq. 5 least squares) */

/* out_dev[0] = sum_i a_i b_i accumulated in FP64 (float32 inputs, n >= 0),
 * deterministic: a fixed grid of blocks writes one FP64 partial each into
 * the caller's workspace `work_dev` (at least spl_dot_f64_workspace_bytes()
 * bytes, device memory owned by the caller), then one block adds the
 * partials in index order.  Calls that share a workspace must not overlap.
 * Errors: SPL_ERR_ARG (NULL pointer, short workspace), SPL_ERR_CUDA. */
long long spl_dot_f64_workspace_bytes(void);
spl_status spl_dot_f64(long long n, const float *a_dev, const float *b_dev, double *out_dev, void *work_dev,
                       long long work_bytes, void *stream);

/* Allocation-free variant of spl_dot_f64, for callers that cannot let a
 * library allocate device memory (frameworks that own all device memory
 * through their own pool, programs with a device-memory budget fixed at
 * start-up, latency-critical loops that cannot afford cudaMalloc's implicit
 * synchronisation).  The paper has no counterpart: this is an interface
 * choice of the library.
 * Same kernels and same result as spl_dot_f64, but the 1024 FP64 partial
 * sums live in a file-scope device array of the library (8 KB, held by every
 * GPU that loads the library until the process exits) instead of a caller
 * workspace.  The first call on a device looks up that array's device
 * address (with the device current) and caches it; make that first call
 * before any stream capture.  The cached address belongs to the device's
 * primary context (the one the CUDA runtime uses): calls under another
 * context, or after cudaDeviceReset, are not supported.  Every call shares
 * the array, which keeps the
 * last call's partials (each call overwrites all of them, nothing needs
 * clearing); calls that overlap on the GPU race on it.
 * n: 0 .. SPL_DOT_NOALLOC_MAX_N elements (the partial count does not depend
 * on n); a longer input is rejected with SPL_ERR_ARG.  Calls no cudaMalloc,
 * cudaFree or allocating routine.  Errors: SPL_ERR_ARG, SPL_ERR_CUDA. */
#define SPL_DOT_NOALLOC_MAX_N (1LL << 40)
spl_status spl_dot_f64_noalloc(long long n, const float *a_dev, const float *b_dev, double *out_dev, void *stream);

/* CGLS updates with FP64 scalars read from device memory (no host sync):
 *   spl_cg_step_x:  x += alpha p;  r -= alpha q;   alpha = num[0] / den[0]
 *   spl_cg_step_p:  p = s + beta p;                beta  = num[0] / den[0]
 * (num, den: FP64 device scalars; den == 0 leaves the vectors unchanged). */
spl_status spl_cg_step_x(long long nx, float *x_dev, const float *p_dev, long long nr, float *r_dev,
                         const float *q_dev, const double *num_dev, const double *den_dev, void *stream);
spl_status spl_cg_step_p(long long n, float *p_dev, const float *s_dev, const double *num_dev,
                         const double *den_dev, void *stream);

/* ---------------------------------------------------------------- misc */

/* FP32 throughput probe (measurement support, no counterpart in the paper):
 * launches blocks_per_sm x (SM count) blocks of 256 threads, each thread
 * running `iters` x 4 x 16 fused multiply-adds on 16 independent chains,
 * as scalar FMAs (packed = 0) or as packed FP32x2 FMAs (packed != 0,
 * __ffma2_rn: two per instruction).  *flop receives the FP32 operation
 * count of the launch (2 per multiply-add), to be divided by the launch's
 * duration measured on `stream`.  out_dev: one float32 of device memory
 * (written only in a case that never happens; it keeps the chains live).
 * Errors: SPL_ERR_ARG, SPL_ERR_CUDA. */
spl_status spl_fp32_probe(int packed, int blocks_per_sm, int iters, float *out_dev, double *flop, void *stream);
/* Number of SMs of the current device. */
int spl_sm_count(void);


/* Message of the last failing call on this thread ("" if none). */
const char *spl_last_error(void);
/* Fault injection for tests: lower the loop bound of the per-cell event
 * loops (and of the per-slab pair enumeration of the learned-footprint
 * projector) to `cap` (1..40; any other value restores the default 40).  With a bound that
 * is too small the kernels stop early, set the geometry's error flag, and
 * spl_geometry_status() reports SPL_ERR_STEPCAP.  Affects launches issued
 * after the call, process-wide.  Returns the previous bound. */
int spl_debug_set_iter_cap(int cap);
/* Library version string. */
const char *spl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPL_H */
