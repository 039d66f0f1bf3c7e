"""Pins of the oracle's footprint-table operator (the splat form: exact
footprints tabulated per parallel view on a grid of step h in an
orthonormal frame of H_w, bilinear interpolation between nodes).

What fixes it without reference to itself: bilinear interpolation
reproduces the exact footprint at every node and is invariant along w (the
footprint is); between nodes it converges to the exact footprint at second
order in h; its matrix is the transpose of its adjoint's; and as h shrinks
the tabulated operator tends to the exact one of Eq. 4."""
import numpy as np
import pytest

from paper_2511_11078_gb300 import inputs as I


def _random_frame(orc, rng):
    w = I.random_directions(rng, 1)[0]
    u = rng.normal(size=3)
    return orc.table_frame(w, u)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_table_is_exact_at_nodes(orc, n):
    rng = np.random.default_rng(4100 + n)
    for _ in range(6):
        w, e1, e2 = _random_frame(orc, rng)
        for h in (1.0 / 8, 1.0 / 32):
            M = orc.table_radius(n, h)
            for _ in range(5):
                i, j = rng.integers(M // 2, 3 * M // 2, size=2)
                p = (i - M) * h * e1 + (j - M) * h * e2
                shift = rng.uniform(-3, 3) * w  # the footprint is invariant along w
                exact = orc.footprint(n, w, p)
                assert abs(orc.table_footprint(n, w, e1, e2, p + shift, h) - exact) <= 1e-12


def test_table_frame_is_orthonormal_and_spans_the_plane(orc):
    rng = np.random.default_rng(4110)
    for _ in range(20):
        w, e1, e2 = _random_frame(orc, rng)
        Q = np.stack([w, e1, e2])
        assert np.allclose(Q @ Q.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(Q) > 0


@pytest.mark.parametrize("n", [2, 3])
def test_table_converges_at_second_order(orc, n):
    """Mean interpolation error over random offsets drops ~4x per halving of h
    (bilinear interpolation of a function with bounded second derivatives)."""
    rng = np.random.default_rng(4120 + n)
    W = 0.5 * (n + 1)
    pts = []
    for _ in range(40):
        w, e1, e2 = _random_frame(orc, rng)
        a, b = rng.uniform(-W, W, size=2)
        pts.append((w, e1, e2, a * e1 + b * e2))
    errs = []
    for h in (1.0 / 8, 1.0 / 16, 1.0 / 32):
        e = [abs(orc.table_footprint(n, w, e1, e2, p, h) - orc.footprint(n, w, p)) for w, e1, e2, p in pts]
        errs.append(np.mean(e))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, (errs, r1, r2)
    # at h = 1/32 the error is a small fraction of the footprint peak
    assert errs[2] < 2e-4 * orc.footprint(n, [0, 0, 1.0], [0, 0, 0])


def _small_parallel(rng, nd=11):
    dirs = np.concatenate([I.random_directions(rng, 3), [[np.cos(0.4), np.sin(0.4), 0.0]]])
    return I.parallel_views(dirs, nd, nd, 1.0, center=(0.21, -0.13, 0.07))


def _oracle_geom(orc, geo):
    return orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u,
                        det_v=geo.det_v, nu=geo.nu, nv=geo.nv)


def test_table_operator_adjointness(orc):
    rng = np.random.default_rng(4130)
    dims = (7, 6, 5)
    origin = I.centred_origin(dims)
    geo = _small_parallel(rng)
    og = _oracle_geom(orc, geo)
    c = rng.normal(size=dims[::-1])
    y = rng.normal(size=geo.n_rays)
    Ac = orc.forward_table(3, dims, origin, c, og)
    ATy = orc.adjoint_table(3, dims, origin, y, og)
    lhs, rhs = float(Ac @ y), float(np.sum(c * ATy))
    assert abs(lhs - rhs) <= 1e-12 * (np.linalg.norm(Ac) * np.linalg.norm(y))


def test_table_operator_tends_to_the_exact_one(orc):
    rng = np.random.default_rng(4140)
    dims = (7, 6, 5)
    origin = I.centred_origin(dims)
    geo = _small_parallel(rng)
    og = _oracle_geom(orc, geo)
    c = rng.uniform(0, 1, size=dims[::-1])
    exact = orc.forward(3, dims, origin, c, og)
    err = []
    for h in (1.0 / 8, 1.0 / 16, 1.0 / 32):
        yt = orc.forward_table(3, dims, origin, c, og, h)
        err.append(np.linalg.norm(yt - exact) / np.linalg.norm(exact))
    assert err[0] > err[1] > err[2] and err[2] < 1e-3, err
