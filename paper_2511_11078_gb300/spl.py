"""Thin ctypes binding of libspl.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; PyTorch only provides
device memory and streams.  If the library is missing, ``lib()`` raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SPL_OK = 0
SPL_RAYS, SPL_PARALLEL, SPL_CONE = 0, 1, 2
SPL_FP_QUAD, SPL_FP_MLP, SPL_FP_DIRECT, SPL_FP_TABLE = 0, 1, 2, 3
SPL_ADJ_AUTO, SPL_ADJ_GATHER, SPL_ADJ_SCATTER = 0, 1, 2
SPL_SEP_AUTO, SPL_SEP_OFF = 0, 1
MLP_PARAMS = 8769
STATUS_NAMES = {0: "SPL_OK", 1: "SPL_ERR_ARG", 2: "SPL_ERR_NONFINITE", 3: "SPL_ERR_CUDA", 4: "SPL_ERR_STEPCAP",
                5: "SPL_ERR_OOM", 6: "SPL_ERR_STATE", 7: "SPL_ERR_UNSUPPORTED", 8: "SPL_ERR_TIMEOUT"}

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_vp = C.c_void_p


class SplError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class GeometryDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("origin", C.c_double * 3),
        ("n_rays", C.c_longlong), ("ray_omega", _dp), ("ray_s", _dp),
        ("n_views", C.c_int), ("view_src", _dp), ("det_center", _dp), ("det_u", _dp), ("det_v", _dp),
        ("nu", C.c_int), ("nv", C.c_int),
    ]


class BasisDesc(C.Structure):
    _fields_ = [("degree", C.c_int), ("mode", C.c_int), ("mlp", _vp), ("kahan", C.c_int), ("adjoint", C.c_int),
                ("separable", C.c_int)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); mirrors include/spl.h
_SIGS = {
    "spl_make_geometry": (C.c_int, [C.POINTER(GeometryDesc), C.POINTER(_vp)]),
    "spl_destroy_geometry": (None, [_vp]),
    "spl_geometry_rays": (C.c_longlong, [_vp]),
    "spl_geometry_coeffs": (C.c_longlong, [_vp]),
    "spl_geometry_status": (C.c_int, [_vp, _vp]),
    "spl_prepare": (C.c_int, [_vp, C.POINTER(BasisDesc), _vp]),
    "spl_forward": (C.c_int, [_vp, C.POINTER(BasisDesc), _vp, _vp, _vp]),
    "spl_adjoint": (C.c_int, [_vp, C.POINTER(BasisDesc), _vp, _vp, _vp]),
    "spl_count_pairs": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "spl_count_pairs_per_ray": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "spl_footprint": (C.c_int, [C.POINTER(BasisDesc), C.c_longlong, _vp, _vp, _vp, _vp]),
    "spl_features": (C.c_int, [C.c_int, C.c_longlong, _vp, _vp, _vp, _vp]),
    "spl_footprint_samples": (C.c_int, [C.c_int, C.c_longlong, _vp, _vp, _vp, _vp, _vp]),
    "spl_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_ulonglong, C.POINTER(_vp)]),
    "spl_mlp_destroy": (None, [_vp]),
    "spl_mlp_degree": (C.c_int, [_vp]),
    "spl_mlp_set_params": (C.c_int, [_vp, _fp]),
    "spl_mlp_get_params": (C.c_int, [_vp, _fp]),
    "spl_mlp_eval": (C.c_int, [_vp, C.c_longlong, _vp, _vp, _vp]),
    "spl_mlp_grad": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "spl_mlp_train_step": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_float, _vp, _vp]),
    "spl_dot_f64_workspace_bytes": (C.c_longlong, []),
    "spl_dot_f64": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp, C.c_longlong, _vp]),
    "spl_dot_f64_noalloc": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp]),
    "spl_cg_step_x": (C.c_int, [C.c_longlong, _vp, _vp, C.c_longlong, _vp, _vp, _vp, _vp, _vp]),
    "spl_cg_step_p": (C.c_int, [C.c_longlong, _vp, _vp, _vp, _vp, _vp]),
    "spl_debug_set_iter_cap": (C.c_int, [C.c_int]),
    "spl_frame": (C.c_int, [C.c_longlong, _dp, _dp, _dp]),
    "spl_mlp_status": (C.c_int, [_vp, _vp]),
    "spl_mlp_save": (C.c_int, [_vp, C.c_char_p]),
    "spl_mlp_load": (C.c_int, [_vp, C.c_char_p]),
    "spl_fp32_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, _dp]),
    "spl_sm_count": (C.c_int, []),
    "spl_last_error": (C.c_char_p, []),
    "spl_version": (C.c_char_p, []),
}


def exported_names():
    return sorted(_SIGS)


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libspl.so (raises if it is absent and not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if build_if_missing:
                    _build.build()
                else:
                    raise RuntimeError("libspl.so is not built (%s); run __graft_entry__.build()" % path)
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(status):
    if status != SPL_OK:
        msg = lib().spl_last_error()
        raise SplError(status, msg.decode() if msg else "")


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (marshalling only)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(a):
    return a.ctypes.data_as(_dp)


class Geometry:
    """Device geometry (spl_make_geometry) for a coefficient grid and a set of
    lines: an inputs.ViewGeometry (parallel / cone views) or an
    inputs.RayGeometry (explicit rays)."""

    def __init__(self, dims, origin, geometry):
        self.dims = tuple(int(v) for v in dims)
        self.origin = np.asarray(origin, dtype=np.float64).reshape(3)
        d = GeometryDesc()
        d.nx, d.ny, d.nz = self.dims
        for e in range(3):
            d.origin[e] = float(self.origin[e])
        keep = []
        if geometry.kind == "rays":
            w = np.ascontiguousarray(geometry.omega, dtype=np.float64)
            s = np.ascontiguousarray(geometry.s, dtype=np.float64)
            keep += [w, s]
            d.kind, d.n_rays, d.ray_omega, d.ray_s = SPL_RAYS, w.shape[0], _dptr(w), _dptr(s)
            self.shape = (w.shape[0],)
        else:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
                    (geometry.src, geometry.det_center, geometry.det_u, geometry.det_v)]
            keep += arrs
            d.kind = SPL_PARALLEL if geometry.kind == "parallel" else SPL_CONE
            d.n_views = arrs[0].shape[0]
            d.view_src, d.det_center, d.det_u, d.det_v = (_dptr(a) for a in arrs)
            d.nu, d.nv = int(geometry.nu), int(geometry.nv)
            self.shape = (d.n_views, d.nv, d.nu)
        self.kind = geometry.kind
        self._prepared = set()
        h = _vp()
        check(lib().spl_make_geometry(C.byref(d), C.byref(h)))
        self._h = h
        self.n_rays = int(lib().spl_geometry_rays(h))
        self.n_coeffs = int(lib().spl_geometry_coeffs(h))

    @property
    def handle(self):
        return self._h

    @property
    def coeff_shape(self):
        return (self.dims[2], self.dims[1], self.dims[0])

    def close(self):
        if getattr(self, "_h", None):
            lib().spl_destroy_geometry(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        check(lib().spl_geometry_status(self._h, _stream(stream)))


def basis(degree: int, mode: int = SPL_FP_QUAD, mlp=None, kahan: bool = True, adjoint: int = SPL_ADJ_AUTO,
          separable: int = SPL_SEP_AUTO) -> BasisDesc:
    b = BasisDesc()
    b.degree, b.mode, b.kahan, b.adjoint = int(degree), int(mode), 1 if kahan else 0, int(adjoint)
    b.separable = int(separable)
    b.mlp = mlp.handle if mlp is not None else None
    return b


def _basis_key(bas: BasisDesc):
    return (int(bas.degree), int(bas.mode), int(bas.separable))


def prepare(geom: Geometry, bas: BasisDesc, stream=None):
    """spl_prepare: build what the projector needs for this basis (the plane
    matrices of slice-separable views, the footprint tables of
    SPL_FP_TABLE); one-time allocation, then a synchronisation."""
    check(lib().spl_prepare(geom.handle, C.byref(bas), _stream(stream)))
    geom._prepared.add(_basis_key(bas))


def _ensure_prepared(geom: Geometry, bas: BasisDesc, stream):
    # spl_forward / spl_adjoint never allocate and refuse a basis whose
    # structures are not built (SPL_ERR_STATE); the binding prepares each
    # (degree, mode, separable) once, before its first use
    if _basis_key(bas) not in geom._prepared:
        prepare(geom, bas, stream)


def forward(geom: Geometry, c, y, bas: BasisDesc, stream=None):
    """y = A c (Algorithm 2).  c: float32 CUDA [nz,ny,nx]; y: float32 CUDA (n_rays)."""
    _check_sizes(geom, c, y)
    _ensure_prepared(geom, bas, stream)
    check(lib().spl_forward(geom.handle, C.byref(bas), _ptr(c), _ptr(y), _stream(stream)))


def adjoint(geom: Geometry, y, c, bas: BasisDesc, stream=None):
    """c = A^T y (matched adjoint)."""
    _check_sizes(geom, c, y)
    _ensure_prepared(geom, bas, stream)
    check(lib().spl_adjoint(geom.handle, C.byref(bas), _ptr(y), _ptr(c), _stream(stream)))


def count_work(geom: Geometry, degree: int, stream=None):
    """(pairs, pieces, flat_pieces) of one forward projection: the
    contributions of Eq. 4 (exact pair count), integrated pieces with the
    full Gauss rule and with the (n+1)-node rule of rays with a zero
    direction component."""
    import torch

    cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
    check(lib().spl_count_pairs(geom.handle, int(degree), _ptr(cnt), _stream(stream)))
    v = cnt.cpu().tolist()
    return int(v[0]), int(v[1]), int(v[2])


def count_pairs(geom: Geometry, degree: int, stream=None) -> int:
    return count_work(geom, degree, stream)[0]


def count_pairs_per_ray(geom: Geometry, degree: int, stream=None):
    """(contributions of each ray as a uint32 CUDA tensor, their total)."""
    import torch

    per = torch.zeros(geom.n_rays, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    check(lib().spl_count_pairs_per_ray(geom.handle, int(degree), _ptr(per), _ptr(tot), _stream(stream)))
    return per, int(tot.item())


def footprint(bas: BasisDesc, omega, p, out, stream=None):
    n = omega.shape[0]
    check(lib().spl_footprint(C.byref(bas), n, _ptr(omega), _ptr(p), _ptr(out), _stream(stream)))


def features(degree: int, omega, p, feat, stream=None):
    check(lib().spl_features(int(degree), omega.shape[0], _ptr(omega), _ptr(p), _ptr(feat), _stream(stream)))


def footprint_samples(degree: int, normals, uniforms, omega, p, stream=None):
    check(lib().spl_footprint_samples(int(degree), normals.shape[0], _ptr(normals), _ptr(uniforms), _ptr(omega),
                                      _ptr(p), _stream(stream)))


class Mlp:
    """The learned footprint f_theta (spl_mlp): 5 -> 64 -> 64 -> 64 -> 1 SiLU."""

    def __init__(self, degree: int, max_batch: int = 8192, seed: int = 0):
        h = _vp()
        check(lib().spl_mlp_create(int(degree), int(max_batch), C.c_ulonglong(int(seed)), C.byref(h)))
        self._h = h
        self.degree = int(degree)
        self.max_batch = int(max_batch)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().spl_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        check(lib().spl_mlp_get_params(self._h, out.ctypes.data_as(_fp)))
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != MLP_PARAMS:
            raise ValueError("need %d parameters" % MLP_PARAMS)
        check(lib().spl_mlp_set_params(self._h, p.ctypes.data_as(_fp)))

    def status(self, stream=None):
        """Synchronise and raise if a tensor-core wait of this network gave up."""
        check(lib().spl_mlp_status(self._h, _stream(stream)))

    def save(self, path: str):
        """spl_mlp_save: parameters, Adam moments and step count to `path`."""
        check(lib().spl_mlp_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        """spl_mlp_load: restore a checkpoint written by save()."""
        check(lib().spl_mlp_load(self._h, os.fsencode(path)))

    def eval(self, feat, out, stream=None):
        check(lib().spl_mlp_eval(self._h, feat.shape[0], _ptr(feat), _ptr(out), _stream(stream)))

    def grad(self, feat, target, grad, loss=None, stream=None):
        check(lib().spl_mlp_grad(self._h, feat.shape[0], _ptr(feat), _ptr(target), _ptr(grad), _ptr(loss),
                                 _stream(stream)))

    def train_step(self, feat, target, lr: float, loss=None, stream=None):
        check(lib().spl_mlp_train_step(self._h, feat.shape[0], _ptr(feat), _ptr(target), C.c_float(lr), _ptr(loss),
                                       _stream(stream)))


def frame(omega):
    """spl_frame: the (u, v) frame of H_w in which the MLP features measure
    offsets, for directions omega [N,3] (host FP64); returns (u, v) [N,3]."""
    w = np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(-1, 3))
    u = np.zeros_like(w)
    v = np.zeros_like(w)
    check(lib().spl_frame(w.shape[0], _dptr(w), _dptr(u), _dptr(v)))
    return u, v


def fp32_probe(out, packed: bool, blocks_per_sm: int = 4, iters: int = 4096, stream=None) -> float:
    """Launch the FP32 FMA throughput probe; returns its FLOP count."""
    flop = C.c_double(0.0)
    check(lib().spl_fp32_probe(1 if packed else 0, int(blocks_per_sm), int(iters), _ptr(out), C.byref(flop),
                               _stream(stream)))
    return float(flop.value)


def sm_count() -> int:
    return int(lib().spl_sm_count())


def dot_workspace(device=None):
    import torch

    nbytes = int(lib().spl_dot_f64_workspace_bytes())
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def dot_f64(a, b, out, work, stream=None):
    """out[0] = sum a_i b_i in FP64 (deterministic)."""
    if a.numel() != b.numel():
        raise ValueError("length mismatch")
    check(lib().spl_dot_f64(a.numel(), _ptr(a), _ptr(b), _ptr(out), _ptr(work), work.numel(), _stream(stream)))


def cg_step_x(x, p, r, q, num, den, stream=None):
    check(lib().spl_cg_step_x(x.numel(), _ptr(x), _ptr(p), r.numel(), _ptr(r), _ptr(q), _ptr(num), _ptr(den),
                              _stream(stream)))


def cg_step_p(p, s, num, den, stream=None):
    check(lib().spl_cg_step_p(p.numel(), _ptr(p), _ptr(s), _ptr(num), _ptr(den), _stream(stream)))


def _check_sizes(geom, c, y):
    import torch

    for t in (c, y):
        if t.dtype != torch.float32:
            raise TypeError("expected float32 tensors")
    if c.numel() != geom.n_coeffs or y.numel() != geom.n_rays:
        raise ValueError("c has %d values (need %d), y has %d (need %d)" % (c.numel(), geom.n_coeffs, y.numel(),
                                                                             geom.n_rays))
