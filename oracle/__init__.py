"""FP64 CPU oracle for the B-spline x-ray transform (SplineSplat, arXiv 2511.11078).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module and this module never imports the product package.

The arithmetic lives in ``oracle.c`` (plain C, double precision).  This file
builds it with gcc on first use and wraps it with ctypes.

Every function cites the passage of the paper it follows:

* ``bspline``      -- the 1-D B-spline generator (Sec. 2.2, tensor-product
                      B-spline basis; Schoenberg's truncated-power formula).
* ``footprint``    -- Pphi(w, p) = int prod_d beta^n(p_d + t w_d) dt, the
                      contribution of Eq. 4, by knot-split Gauss-Legendre.
* ``forward``      -- Eq. 4 summed over the exact pair set (route A).
* ``adjoint``      -- transpose of the matrix of Eq. 6.
* ``forward_segmented`` -- Eq. 2 applied to Eq. 3 directly (route B).
* ``siddon``       -- voxel path lengths, the classic DDA of Sec. 1.
* ``dda_visit``    -- Algorithm 2 + Algorithm 3 enumeration (set check only).
* ``mlp_forward`` / ``mlp_loss_grad`` -- the MLP f_theta of Sec. 2.2 and the
                      gradient of the L2 loss of Algorithm 1.
* ``features``     -- MLP input features (signed-permutation chamber + frame
                      u perpendicular to w, v = u x w of Algorithm 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_llp = C.POINTER(C.c_longlong)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("n_views", C.c_int), ("nu", C.c_int), ("nv", C.c_int),
        ("n_rays", C.c_longlong),
        ("ray_w", _dp), ("ray_s", _dp),
        ("dir_or_src", _dp), ("det_c", _dp), ("det_u", _dp), ("det_v", _dp),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_bspline.restype = C.c_double
            lib.orc_bspline.argtypes = [C.c_int, C.c_double]
            lib.orc_gauss_legendre.argtypes = [C.c_int, _dp, _dp]
            lib.orc_gl_order.argtypes = [C.c_int]
            lib.orc_footprint.restype = C.c_double
            lib.orc_footprint.argtypes = [C.c_int, _dp, _dp]
            lib.orc_footprint_m.restype = C.c_double
            lib.orc_footprint_m.argtypes = [C.c_int, _dp, _dp, C.c_int]
            lib.orc_footprint_batch.argtypes = [C.c_int, C.c_longlong, _dp, _dp, _dp]
            G = C.POINTER(_Geom)
            lib.orc_geom_rays.restype = C.c_longlong
            lib.orc_geom_rays.argtypes = [G]
            lib.orc_geom_all_rays.argtypes = [G, _dp, _dp]
            lib.orc_forward.argtypes = [C.c_int, _ip, _dp, _dp, G, _dp, C.c_int]
            lib.orc_forward_subset.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_longlong, _llp, _dp, _llp, C.c_int]
            lib.orc_count_pairs.restype = C.c_longlong
            lib.orc_count_pairs.argtypes = [C.c_int, _ip, _dp, G, _llp]
            lib.orc_adjoint.argtypes = [C.c_int, _ip, _dp, _dp, G, _dp]
            lib.orc_adjoint_at.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_longlong, _llp, _dp, _llp, C.c_int]
            lib.orc_adjoint_subset.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_longlong, _llp, _dp, _llp, C.c_int]
            lib.orc_adjoint_at_views.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_longlong, _llp, _dp, _llp, C.c_int]
            lib.orc_forward_segmented.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_longlong, _llp, _dp, C.c_int]
            lib.orc_eval_spline.restype = C.c_double
            lib.orc_eval_spline.argtypes = [C.c_int, _ip, _dp, _dp, _dp]
            lib.orc_siddon.argtypes = [_ip, _dp, _dp, G, _dp]
            lib.orc_dda_visit.restype = C.c_longlong
            lib.orc_dda_visit.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp, _llp, C.c_longlong, _ip, _llp]
            lib.orc_bf16_round.restype = C.c_double
            lib.orc_bf16_round.argtypes = [C.c_double]
            lib.orc_mlp_param_count.restype = C.c_longlong
            lib.orc_mlp_param_count.argtypes = [C.c_int, _ip]
            lib.orc_mlp_forward.argtypes = [C.c_int, _ip, _dp, C.c_longlong, _dp, _dp, C.c_int]
            lib.orc_mlp_flip_variants.restype = C.c_longlong
            lib.orc_mlp_flip_variants.argtypes = [C.c_int, _ip, _dp, _dp, C.c_double, _dp, C.c_longlong]
            lib.orc_mlp_loss_grad.restype = C.c_double
            lib.orc_mlp_loss_grad.argtypes = [C.c_int, _ip, _dp, C.c_longlong, _dp, _dp, _dp]
            lib.orc_mlp_loss_grad_mode.restype = C.c_double
            lib.orc_mlp_loss_grad_mode.argtypes = [C.c_int, _ip, _dp, C.c_longlong, _dp, _dp, _dp, C.c_int]
            lib.orc_features.argtypes = [C.c_int, _dp, _dp, _dp]
            lib.orc_forward_mlp.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_int, _ip, _dp, C.c_int, _dp]
            lib.orc_num_threads.restype = C.c_int
            lib.orc_table_radius.restype = C.c_int
            lib.orc_table_radius.argtypes = [C.c_int, C.c_double]
            lib.orc_table_frame.argtypes = [_dp, _dp, _dp, _dp, _dp]
            lib.orc_table_footprint.restype = C.c_double
            lib.orc_table_footprint.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, _dp]
            lib.orc_forward_table.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_double, _dp]
            lib.orc_adjoint_table.argtypes = [C.c_int, _ip, _dp, _dp, G, C.c_double, _dp]
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _ll(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_llp)


class Geometry:
    """FP64 ray geometry (Eq. 1) built from plain arrays.

    kind "rays":     omega [R,3], s [R,3]
    kind "parallel": view direction [V,3], detector centre/u/v [V,3], nu, nv
    kind "cone":     source [V,3],        detector centre/u/v [V,3], nu, nv
    Ray r = (view * nv + iv) * nu + iu, pixel centre
    det_center + (iu - (nu-1)/2) det_u + (iv - (nv-1)/2) det_v.
    """

    def __init__(self, kind, **kw):
        self.kind = kind
        self._keep = []
        g = _Geom()
        if kind == "rays":
            w, wp = _d(kw["omega"])
            s, sp = _d(kw["s"])
            g.kind, g.n_rays, g.ray_w, g.ray_s = 0, w.shape[0], wp, sp
            self._keep += [w, s]
            self.n_rays = w.shape[0]
        else:
            src = kw["direction"] if kind == "parallel" else kw["source"]
            a, ap = _d(src)
            c, cp = _d(kw["det_center"])
            u, up = _d(kw["det_u"])
            v, vp = _d(kw["det_v"])
            g.kind = 1 if kind == "parallel" else 2
            g.n_views, g.nu, g.nv = a.shape[0], int(kw["nu"]), int(kw["nv"])
            g.dir_or_src, g.det_c, g.det_u, g.det_v = ap, cp, up, vp
            self._keep += [a, c, u, v]
            self.n_rays = a.shape[0] * int(kw["nu"]) * int(kw["nv"])
        self._g = g

    @property
    def ptr(self):
        return C.byref(self._g)

    def rays(self):
        """All rays as (s [R,3], omega [R,3]) in FP64."""
        s = np.zeros((self.n_rays, 3))
        w = np.zeros((self.n_rays, 3))
        _load().orc_geom_all_rays(self.ptr, s.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
        return s, w


def num_threads() -> int:
    return int(_load().orc_num_threads())


def bspline(n: int, x):
    """beta^n(x) (Sec. 2.2), vectorised over x."""
    lib = _load()
    x = np.asarray(x, dtype=np.float64)
    return np.vectorize(lambda v: lib.orc_bspline(int(n), float(v)), otypes=[np.float64])(x)


def gauss_legendre(m: int):
    x = np.zeros(m)
    w = np.zeros(m)
    rc = _load().orc_gauss_legendre(int(m), x.ctypes.data_as(_dp), w.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError("unsupported Gauss-Legendre order %d" % m)
    return x, w


def gl_order(n: int) -> int:
    return int(_load().orc_gl_order(int(n)))


def footprint(n: int, omega, p, m: int | None = None) -> float:
    """Exact Pphi(omega, p) (Eq. 2 applied to phi, the contribution of Eq. 4)."""
    w, wp = _d(np.asarray(omega, dtype=np.float64).reshape(3))
    q, qp = _d(np.asarray(p, dtype=np.float64).reshape(3))
    lib = _load()
    if m is None:
        return float(lib.orc_footprint(int(n), wp, qp))
    return float(lib.orc_footprint_m(int(n), wp, qp, int(m)))


def footprint_batch(n: int, omega, p):
    w, wp = _d(np.asarray(omega).reshape(-1, 3))
    q, qp = _d(np.asarray(p).reshape(-1, 3))
    out = np.zeros(w.shape[0])
    _load().orc_footprint_batch(int(n), w.shape[0], wp, qp, out.ctypes.data_as(_dp))
    return out


def _grid(dims, origin):
    d, dp = _i(np.asarray(dims).reshape(3))
    o, op = _d(np.asarray(origin, dtype=np.float64).reshape(3))
    return (d, o), dp, op


def forward(n, dims, origin, c, geom: Geometry, nthreads: int = 0):
    """y = A c with A from Eq. 6 (route A: sum over the exact pair set)."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    y = np.zeros(geom.n_rays)
    _load().orc_forward(int(n), dp, op, cp, geom.ptr, y.ctypes.data_as(_dp), int(nthreads))
    return y


def forward_subset(n, dims, origin, c, geom: Geometry, rays, nthreads: int = 0):
    """Rows `rays` of A c; also returns the number of pairs per ray."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    r, rp = _ll(rays)
    y = np.zeros(r.shape[0])
    pairs = np.zeros(r.shape[0], dtype=np.int64)
    _load().orc_forward_subset(int(n), dp, op, cp, geom.ptr, r.shape[0], rp, y.ctypes.data_as(_dp),
                               pairs.ctypes.data_as(_llp), int(nthreads))
    return y, pairs


def count_pairs(n, dims, origin, geom: Geometry, per_ray: bool = False):
    keep, dp, op = _grid(dims, origin)
    if per_ray:
        pr = np.zeros(geom.n_rays, dtype=np.int64)
        tot = _load().orc_count_pairs(int(n), dp, op, geom.ptr, pr.ctypes.data_as(_llp))
        return int(tot), pr
    return int(_load().orc_count_pairs(int(n), dp, op, geom.ptr, None))


def adjoint(n, dims, origin, y, geom: Geometry):
    """c = A^T y (transpose of Eq. 6), overwrites."""
    keep, dp, op = _grid(dims, origin)
    yy, yp = _d(np.asarray(y).reshape(-1))
    c = np.zeros(int(np.prod(dims)))
    _load().orc_adjoint(int(n), dp, op, yp, geom.ptr, c.ctypes.data_as(_dp))
    return c.reshape(int(dims[2]), int(dims[1]), int(dims[0]))


def adjoint_at(n, dims, origin, y, geom: Geometry, kidx, nthreads: int = 0):
    """Entries `kidx` (linear indices) of A^T y; also the pair count of each."""
    keep, dp, op = _grid(dims, origin)
    yy, yp = _d(np.asarray(y).reshape(-1))
    k, kp = _ll(kidx)
    out = np.zeros(k.shape[0])
    pairs = np.zeros(k.shape[0], dtype=np.int64)
    _load().orc_adjoint_at(int(n), dp, op, yp, geom.ptr, k.shape[0], kp, out.ctypes.data_as(_dp),
                           pairs.ctypes.data_as(_llp), int(nthreads))
    return out, pairs


def adjoint_at_views(n, dims, origin, y, geom: Geometry, kidx, nthreads: int = 0):
    """Entries `kidx` of A^T y for a view geometry, visiting per view only
    the detector window of each coefficient's support (the same sum as
    adjoint_at, fast enough for full-size detectors)."""
    if geom.kind == "rays":
        raise ValueError("adjoint_at_views needs a view geometry")
    keep, dp, op = _grid(dims, origin)
    yy, yp = _d(np.asarray(y).reshape(-1))
    k, kp = _ll(kidx)
    out = np.zeros(k.shape[0])
    pairs = np.zeros(k.shape[0], dtype=np.int64)
    _load().orc_adjoint_at_views(int(n), dp, op, yp, geom.ptr, k.shape[0], kp, out.ctypes.data_as(_dp),
                                 pairs.ctypes.data_as(_llp), int(nthreads))
    return out, pairs


def adjoint_subset(n, dims, origin, y, geom: Geometry, rays, nthreads: int = 0):
    """sum over the listed rays of y_i times their rows of Eq. 6 (transpose):
    returns (c [nz,ny,nx], number of pairs)."""
    keep, dp, op = _grid(dims, origin)
    yy, yp = _d(np.asarray(y).reshape(-1))
    r, rp = _ll(rays)
    c = np.zeros(int(np.prod(dims)))
    np_ = np.zeros(1, dtype=np.int64)
    _load().orc_adjoint_subset(int(n), dp, op, yp, geom.ptr, r.shape[0], rp, c.ctypes.data_as(_dp),
                               np_.ctypes.data_as(_llp), int(nthreads))
    return c.reshape(int(dims[2]), int(dims[1]), int(dims[0])), int(np_[0])


def forward_segmented(n, dims, origin, c, geom: Geometry, rays=None, nthreads: int = 0):
    """Route B: Eq. 2 of Eq. 3 split at every knot plane (all rays or a subset)."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    lib = _load()
    if rays is None:
        y = np.zeros(geom.n_rays)
        lib.orc_forward_segmented(int(n), dp, op, cp, geom.ptr, 0, None, y.ctypes.data_as(_dp), int(nthreads))
        return y
    r, rp = _ll(rays)
    y = np.zeros(r.shape[0])
    lib.orc_forward_segmented(int(n), dp, op, cp, geom.ptr, r.shape[0], rp, y.ctypes.data_as(_dp), int(nthreads))
    return y


def eval_spline(n, dims, origin, c, x):
    """f(x) of Eq. 3 at one point."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    xx, xp = _d(np.asarray(x).reshape(3))
    return float(_load().orc_eval_spline(int(n), dp, op, cp, xp))


def siddon(dims, origin, c, geom: Geometry):
    """Voxel path-length projector (Siddon), the classic DDA of Sec. 1."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    y = np.zeros(geom.n_rays)
    _load().orc_siddon(dp, op, cp, geom.ptr, y.ctypes.data_as(_dp))
    return y


def dda_visit(n, R, dims, origin, s, omega, cap: int = 1 << 20):
    """Algorithm 2 + 3 enumeration for one ray: (visited linear indices,
    max cells per dominant-axis slab, number of DDA cells)."""
    keep, dp, op = _grid(dims, origin)
    ss, sp = _d(np.asarray(s).reshape(3))
    ww, wp = _d(np.asarray(omega).reshape(3))
    out = np.zeros(cap, dtype=np.int64)
    mc = C.c_int(0)
    nc = C.c_longlong(0)
    cnt = _load().orc_dda_visit(int(n), int(R), dp, op, sp, wp, out.ctypes.data_as(_llp), cap,
                                C.byref(mc), C.byref(nc))
    if cnt < 0:
        raise RuntimeError("dda_visit: capacity exceeded")
    return out[:cnt].copy(), int(mc.value), int(nc.value)


def bf16_round(x: float) -> float:
    return float(_load().orc_bf16_round(float(x)))


def mlp_param_count(sizes) -> int:
    s, sp = _i(sizes)
    return int(_load().orc_mlp_param_count(len(sizes) - 1, sp))


def mlp_forward(sizes, params, X, mode: int = 0):
    """f_theta(X) for a batch; mode 0 FP64, 1 BF16 contract, 2 split-BF16."""
    s, sp = _i(sizes)
    p, pp = _d(params)
    x, xp = _d(np.asarray(X).reshape(-1, sizes[0]))
    out = np.zeros(x.shape[0])
    _load().orc_mlp_forward(len(sizes) - 1, sp, pp, x.shape[0], xp, out.ctypes.data_as(_dp), int(mode))
    return out


def mlp_flip_variants(sizes, params, x, rel_eps: float, cap: int = 4096):
    """Outputs of the BF16 contract for one feature row x with a single
    hidden activation that lies within rel_eps of a BF16 rounding boundary
    rounded the other way (one value per such activation and direction)."""
    s, sp = _i(sizes)
    p, pp = _d(params)
    xx, xp = _d(np.asarray(x).reshape(-1))
    out = np.zeros(cap)
    n = _load().orc_mlp_flip_variants(len(sizes) - 1, sp, pp, xp, float(rel_eps), out.ctypes.data_as(_dp), cap)
    return out[:min(n, cap)].copy()


def mlp_loss_grad(sizes, params, X, Y, mode: int = 0):
    """(L, dL/dparams) for L = mean (f_theta(x) - y)^2 (Algorithm 1's loss);
    mode 1 differentiates the BF16-contract forward (roundings passed
    straight through)."""
    s, sp = _i(sizes)
    p, pp = _d(params)
    x, xp = _d(np.asarray(X).reshape(-1, sizes[0]))
    yy, yp = _d(np.asarray(Y).reshape(-1))
    g = np.zeros(p.shape[0])
    loss = _load().orc_mlp_loss_grad_mode(len(sizes) - 1, sp, pp, x.shape[0], xp, yp, g.ctypes.data_as(_dp),
                                          int(mode))
    return float(loss), g


def features(n, omega, p):
    """MLP input features for one (omega, p)."""
    w, wp = _d(np.asarray(omega).reshape(3))
    q, qp = _d(np.asarray(p).reshape(3))
    f = np.zeros(5)
    _load().orc_features(int(n), wp, qp, f.ctypes.data_as(_dp))
    return f


def forward_mlp(n, dims, origin, c, geom: Geometry, sizes, params, mode: int = 1):
    """Algorithm 2 with f_theta in place of Pphi, over the exact pair set."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    s, sp = _i(sizes)
    p, pp = _d(params)
    y = np.zeros(geom.n_rays)
    _load().orc_forward_mlp(int(n), dp, op, cp, geom.ptr, len(sizes) - 1, sp, pp, int(mode), y.ctypes.data_as(_dp))
    return y


# ---------------------------------------------------------------- footprint tables (splat form)
TABLE_STEP = 1.0 / 32.0


def table_radius(n, h=TABLE_STEP) -> int:
    """M: the table nodes are (i - M) h e1 + (j - M) h e2, i, j = 0..2M."""
    return int(_load().orc_table_radius(int(n), float(h)))


def table_frame(direction, det_u):
    """(w, e1, e2): unit direction and the orthonormal frame of H_w."""
    d, dp = _d(np.asarray(direction).reshape(3))
    u, up = _d(np.asarray(det_u).reshape(3))
    w, e1, e2 = np.zeros(3), np.zeros(3), np.zeros(3)
    _load().orc_table_frame(dp, up, w.ctypes.data_as(_dp), e1.ctypes.data_as(_dp), e2.ctypes.data_as(_dp))
    return w, e1, e2


def table_footprint(n, w, e1, e2, p, h=TABLE_STEP) -> float:
    """Bilinear interpolation of the exact-footprint table at offset p."""
    args = [_d(np.asarray(a).reshape(3)) for a in (w, e1, e2, p)]
    return float(_load().orc_table_footprint(int(n), args[0][1], args[1][1], args[2][1], float(h), args[3][1]))


def forward_table(n, dims, origin, c, geom: Geometry, h=TABLE_STEP):
    """y = A_T c: the exact pairs with tabulated footprints (parallel views)."""
    keep, dp, op = _grid(dims, origin)
    cc, cp = _d(c.reshape(-1))
    y = np.zeros(geom.n_rays)
    _load().orc_forward_table(int(n), dp, op, cp, geom.ptr, float(h), y.ctypes.data_as(_dp))
    return y


def adjoint_table(n, dims, origin, y, geom: Geometry, h=TABLE_STEP):
    """c = A_T^T y."""
    keep, dp, op = _grid(dims, origin)
    yy, yp = _d(np.asarray(y).reshape(-1))
    c = np.zeros(int(np.prod(dims)))
    _load().orc_adjoint_table(int(n), dp, op, yp, geom.ptr, float(h), c.ctypes.data_as(_dp))
    return c.reshape(int(dims[2]), int(dims[1]), int(dims[0]))
