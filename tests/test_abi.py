"""C-ABI boundary checks that need no GPU: the library builds and loads,
exports every function include/spl.h declares, and rejects bad descriptors
on the host before touching the device."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def spl():
    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import spl as S

    B.build()
    S.lib()
    return S


def declared_functions():
    src = open(os.path.join(ROOT, "include", "spl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(spl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("spl_make_geometry", "spl_forward", "spl_adjoint", "spl_footprint"):
        assert required in names


def test_library_exports_every_declared_symbol(spl):
    L = C.CDLL(spl.lib_path())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    # the binding wraps every declared function and nothing else
    assert set(spl.exported_names()) == set(declared_functions())


def test_version(spl):
    assert b"sm_103a" in spl.lib().spl_version()


def _desc(spl, kind, **kw):
    d = spl.GeometryDesc()
    d.kind = kind
    d.nx = kw.get("nx", 4)
    d.ny = kw.get("ny", 4)
    d.nz = kw.get("nz", 4)
    return d


def _make(spl, d):
    h = C.c_void_p()
    st = spl.lib().spl_make_geometry(C.byref(d), C.byref(h))
    return st, h


def test_rejects_nonfinite_and_zero_rays(spl):
    for w, s, code in [([[math.nan, 0, 1]], [[0, 0, 0]], 2), ([[0, 0, 0]], [[0, 0, 0]], 2),
                       ([[0, 0, 1]], [[math.inf, 0, 0]], 2)]:
        w = np.asarray(w, dtype=np.float64)
        s = np.asarray(s, dtype=np.float64)
        d = _desc(spl, spl.SPL_RAYS)
        d.n_rays, d.ray_omega, d.ray_s = 1, spl._dptr(w), spl._dptr(s)
        st, h = _make(spl, d)
        assert st == code and not h.value
        assert spl.lib().spl_last_error()


def test_rejects_bad_grid_and_kind(spl):
    st, _ = _make(spl, _desc(spl, spl.SPL_RAYS, nx=0))
    assert st == 7
    st, _ = _make(spl, _desc(spl, spl.SPL_RAYS, nx=4096))
    assert st == 7
    st, _ = _make(spl, _desc(spl, 9))
    assert st == 1


def test_rejects_degenerate_views(spl):
    one = np.array([[0.0, 0.0, 1.0]])
    z = np.zeros((1, 3))
    ex = np.array([[1.0, 0, 0]])
    d = _desc(spl, spl.SPL_PARALLEL)
    d.n_views, d.nu, d.nv = 1, 4, 4
    # detector axes parallel
    d.view_src, d.det_center, d.det_u, d.det_v = spl._dptr(one), spl._dptr(z), spl._dptr(ex), spl._dptr(ex)
    st, _ = _make(spl, d)
    assert st == 2
    # direction lying in the detector plane
    ey = np.array([[0.0, 1.0, 0]])
    d.view_src, d.det_u, d.det_v = spl._dptr(ex), spl._dptr(ex), spl._dptr(ey)
    st, _ = _make(spl, d)
    assert st == 1
    # zero pixels
    d.nu = 0
    st, _ = _make(spl, d)
    assert st == 1


def test_null_arguments_are_rejected(spl):
    L = spl.lib()
    b = spl.basis(3)
    assert L.spl_forward(None, C.byref(b), None, None, None) == 1
    assert L.spl_adjoint(None, C.byref(b), None, None, None) == 1
    bad = spl.basis(5)
    assert L.spl_footprint(C.byref(bad), 1, None, None, None, None) == 1
    assert L.spl_dot_f64(4, None, None, None, None, 0, None) == 1
    assert L.spl_count_pairs(None, 3, None, None) == 1
    assert L.spl_prepare(None, C.byref(b), None) == 1
    assert L.spl_features(7, 1, None, None, None, None) == 1


def test_basis_modes_are_validated_on_the_host(spl):
    """Every footprint mode the header names passes the descriptor check
    (count 0: no device work); unknown modes and separable settings fail."""
    L = spl.lib()
    for mode in (spl.SPL_FP_QUAD, spl.SPL_FP_DIRECT, spl.SPL_FP_TABLE):
        b = spl.basis(3, mode)
        assert L.spl_footprint(C.byref(b), 0, None, None, None, None) == 0
    bad = spl.basis(3)
    bad.mode = 9
    assert L.spl_footprint(C.byref(bad), 0, None, None, None, None) == 1
    bad = spl.basis(3, separable=7)
    assert L.spl_footprint(C.byref(bad), 0, None, None, None, None) == 1
    mlp_without_net = spl.basis(3, spl.SPL_FP_MLP)
    assert L.spl_footprint(C.byref(mlp_without_net), 0, None, None, None, None) == 1


def test_frame_is_the_feature_frame(spl, orc):
    """spl_frame (a host call) returns the frame of H_w in which the MLP
    features measure offsets: orthonormal, perpendicular to w, and the
    oracle's features 4 and 5 of (w, p) are <p, u> sqrt(3)/W and
    <p, v> sqrt(3)/W (the oracle computes them from the chamber frame of its
    own, independently written canonicalisation)."""
    rng = np.random.default_rng(404)
    w = rng.normal(size=(300, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    # directions on chamber walls and ties, axis-aligned, negative zeros
    extra = np.array([[0, 0, 1.0], [0, 1.0, 0], [-1.0, 0, 0], [1, 1, 0], [1, 1, 1], [-1, 1, -1], [0, -1, 1],
                      [1e-12, 0.3, -0.9], [0.5, 0.5, -0.70710678118654757]])
    extra /= np.linalg.norm(extra, axis=1, keepdims=True)
    w = np.concatenate([w, extra])
    u, v = spl.frame(w)
    np.testing.assert_allclose(np.sum(u * u, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.sum(v * v, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(np.sum(u * v, axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose(np.sum(u * w, axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose(np.sum(v * w, axis=1), 0.0, atol=1e-14)
    # v = +-(u x w): the sign is the determinant of the direction's signed permutation
    np.testing.assert_allclose(np.abs(np.sum(v * np.cross(u, w), axis=1)), 1.0, atol=1e-14)
    for n in (1, 3):
        sc = np.sqrt(3.0) / (0.5 * (n + 1))
        for i in range(0, w.shape[0], 7):
            p = rng.normal(size=3) * 2.0
            f = orc.features(n, w[i], p)
            assert abs(f[3] - np.dot(p, u[i]) * sc) <= 1e-12
            assert abs(f[4] - np.dot(p, v[i]) * sc) <= 1e-12
    # the frame does not depend on the length of w; zero directions are refused
    u2, v2 = spl.frame(3.5 * w[:5])
    np.testing.assert_allclose(u2, u[:5], atol=1e-15)
    np.testing.assert_allclose(v2, v[:5], atol=1e-15)
    z = np.zeros((1, 3))
    st = spl.lib().spl_frame(1, spl._dptr(z), spl._dptr(np.zeros((1, 3))), spl._dptr(np.zeros((1, 3))))
    assert st == 2
