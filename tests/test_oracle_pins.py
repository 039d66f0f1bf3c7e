"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (tests/golden), textbook formulas (tests/textbook.py), an independent
exact route, brute force on tiny inputs, or invariants of the x-ray
transform (Eq. 2-4), chosen so that a dropped term, a wrong sign or index, or
a transposed operand fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import textbook as TB
from paper_2511_11078_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# 1-D B-spline (Sec. 2.2) and the quadrature rule
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_bspline_matches_textbook_piecewise_form(orc, n):
    x = np.linspace(-3, 3, 1201)
    x = np.concatenate([x, [-0.5, 0.5, -1.5, 1.5, -2.0, 2.0, -1.0, 1.0]])
    np.testing.assert_allclose(orc.bspline(n, x), TB.bspline(n, x), rtol=0, atol=2e-15)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_bspline_centred_recurrence(orc, n):
    # beta^n(x) = ((W + x) beta^{n-1}(x + 1/2) + (W - x) beta^{n-1}(x - 1/2)) / n
    W = 0.5 * (n + 1)
    x = np.random.default_rng(3).uniform(-W - 0.3, W + 0.3, 400)
    lhs = orc.bspline(n, x)
    rhs = ((W + x) * orc.bspline(n - 1, x + 0.5) + (W - x) * orc.bspline(n - 1, x - 0.5)) / n
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_bspline_partition_of_unity_and_mass(orc, n):
    x = np.random.default_rng(4).uniform(-5, 5, 200)
    s = sum(orc.bspline(n, x - k) for k in range(-8, 9))
    np.testing.assert_allclose(s, 1.0, atol=1e-14)
    # unit mass: integrate each unit piece with the exact rule
    W = 0.5 * (n + 1)
    gx, gw = orc.gauss_legendre(max(1, n + 1))
    tot = 0.0
    for a in np.arange(-W, W, 1.0):
        tot += 0.5 * np.sum(gw * orc.bspline(n, a + 0.5 + 0.5 * gx))
    assert abs(tot - 1.0) < 1e-14


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 12])
def test_gauss_legendre_exactness(orc, m):
    x, w = orc.gauss_legendre(m)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * m):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, (m, k)
    # not exact one degree higher (x^(2m) has a nonzero error)
    assert abs(np.sum(w * x ** (2 * m)) - 2.0 / (2 * m + 1)) > 1e-10


def test_gl_order_is_minimal_exact(orc):
    for n in range(4):
        m = orc.gl_order(n)
        assert 2 * m - 1 >= 3 * n and (m == 1 or 2 * (m - 1) - 1 < 3 * n)


# --------------------------------------------------------------------------
# exact footprint Pphi(w, p) (Eq. 2 / Eq. 4)
# --------------------------------------------------------------------------
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "footprint_closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t = line.split()
            rows.append((int(t[0]), [float(v) for v in t[1:4]], [float(v) for v in t[4:7]], float(t[7])))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_footprint_golden_closed_forms(orc, row):
    n, w, p, val = row
    w = np.asarray(w)
    w = w / np.linalg.norm(w)
    got = orc.footprint(n, w, p)
    assert abs(got - val) <= 1e-14 * max(1.0, abs(val)), (row, got)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_footprint_axis_aligned_is_2d_tensor_bspline(orc, n):
    rng = np.random.default_rng(10 + n)
    for d in range(3):
        w = np.zeros(3)
        w[d] = 1.0 if d != 1 else -1.0
        for _ in range(40):
            p = rng.uniform(-2.5, 2.5, 3)
            a, b = [e for e in range(3) if e != d]
            ref = TB.bspline(n, p[a]) * TB.bspline(n, p[b])
            assert abs(orc.footprint(n, w, p) - ref) < 1e-14


def test_footprint_degree0_is_cube_chord(orc):
    rng = np.random.default_rng(11)
    for _ in range(300):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        p = rng.uniform(-0.9, 0.9, 3)
        ref = TB.box_chord([-0.5] * 3, [0.5] * 3, p, w)
        assert abs(orc.footprint(0, w, p) - ref) < 1e-13


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_footprint_symmetries(orc, n):
    rng = np.random.default_rng(20 + n)
    for _ in range(60):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        p = rng.uniform(-1.8, 1.8, 3)
        ref = orc.footprint(n, w, p)
        tol = 1e-14 * max(1.0, abs(ref))
        assert abs(orc.footprint(n, -w, p) - ref) < tol
        if n > 0:  # beta^0 is half-open: p -> -p only holds off the faces
            assert abs(orc.footprint(n, w, -p) - ref) < tol
        assert abs(orc.footprint(n, w, p + rng.uniform(-7, 7) * w) - ref) < 1e-13
        perm = rng.permutation(3)
        sg = rng.choice([-1.0, 1.0], 3) if n > 0 else np.ones(3)
        assert abs(orc.footprint(n, sg * w[perm], sg * p[perm]) - ref) < tol
        # more quadrature nodes than needed give the same value (exactness)
        assert abs(orc.footprint(n, w, p, m=orc.gl_order(n) + 4) - ref) < tol


@pytest.mark.parametrize("n", [2, 3])
def test_footprint_unit_mass_over_plane(orc, n):
    # int_{H_w} Pphi(w, p) dp = int phi = 1 (Fubini); fine trapezoid grid
    W = 0.5 * (n + 1)
    rng = np.random.default_rng(30 + n)
    R = math.sqrt(3.0) * W + 0.05
    k = 161
    g = np.linspace(-R, R, k)
    h = g[1] - g[0]
    for _ in range(2):
        w = rng.normal(size=3)
        w /= np.linalg.norm(w)
        u, v = I.detector_frame(w)
        A, B = np.meshgrid(g, g, indexing="ij")
        P = A.reshape(-1, 1) * u + B.reshape(-1, 1) * v
        vals = orc.footprint_batch(n, np.tile(w, (P.shape[0], 1)), P)
        assert abs(vals.sum() * h * h - 1.0) < 1e-6


# --------------------------------------------------------------------------
# the transform: route A (Eq. 4) against independent routes
# --------------------------------------------------------------------------
def _random_rays_through(rng, count, dims, origin, spread=0.5):
    ctr = origin + (np.asarray(dims) - 1) / 2.0
    w = I.random_directions(rng, count)
    s = np.zeros((count, 3))
    ext = np.asarray(dims) * spread
    for i in range(count):
        s[i] = ctr + rng.uniform(-1, 1, 3) * ext + rng.uniform(-20, 20) * w[i]
    return w, s


@pytest.mark.parametrize("n", [1, 2, 3])
def test_route_a_equals_route_b(orc, n):
    rng = np.random.default_rng(40 + n)
    dims = (9, 8, 7)
    origin = np.array([0.3, -2.0, 1.7])
    c = rng.normal(size=(7, 8, 9))
    w, s = _random_rays_through(rng, 60, dims, origin)
    g = orc.Geometry("rays", omega=w, s=s)
    ya = orc.forward(n, dims, origin, c, g)
    yb = orc.forward_segmented(n, dims, origin, c, g)
    assert np.max(np.abs(ya - yb)) <= 1e-12 * np.max(np.abs(ya))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_route_a_brute_force_midpoint(orc, n):
    rng = np.random.default_rng(50 + n)
    dims = (6, 5, 4)
    origin = np.array([-2.5, -2.0, -1.5])
    c = rng.uniform(-1, 1, size=(4, 5, 6))
    w, s = _random_rays_through(rng, 4, dims, origin, spread=0.3)
    g = orc.Geometry("rays", omega=w, s=s)
    ya = orc.forward(n, dims, origin, c, g)
    W = 0.5 * (n + 1)
    lo = origin - W
    hi = origin + np.asarray(dims) - 1 + W
    h = 1e-4
    for i in range(len(ya)):
        # parameter range of the ray inside the dilated box
        t0, t1 = -np.inf, np.inf
        for d in range(3):
            a, b = (lo[d] - s[i, d]) / w[i, d], (hi[d] - s[i, d]) / w[i, d]
            t0, t1 = max(t0, min(a, b)), min(t1, max(a, b))
        nseg = int(np.ceil((t1 - t0) / h))
        hh = (t1 - t0) / nseg
        tot = 0.0
        for chunk in np.array_split(np.arange(nseg), max(1, nseg // 50000)):
            t = t0 + (chunk + 0.5) * hh
            X = s[i] + t[:, None] * w[i]
            tot += TB.spline_on_points(n, c, origin, X).sum() * hh
        assert abs(tot - ya[i]) <= 1e-7 * max(1.0, abs(ya[i])), (i, tot, ya[i])


def test_one_hot_coefficient_placement(orc):
    # anisotropic grid, one nonzero coefficient, axis-aligned ray through its
    # centre: y = beta(0)^2 only if the index -> position map is right
    dims = (7, 5, 4)
    origin = np.array([1.0, -3.0, 10.0])
    n = 3
    for (kx, ky, kz) in [(5, 1, 2), (0, 4, 3), (6, 0, 0)]:
        c = np.zeros((4, 5, 7))
        c[kz, ky, kx] = 1.0
        pos = origin + np.array([kx, ky, kz])
        rays_w = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [0, 0, 1.0]])
        rays_s = np.array([pos, pos, pos, pos + np.array([1.0, 0, 0])])
        g = orc.Geometry("rays", omega=rays_w, s=rays_s)
        y = orc.forward(n, dims, origin, c, g)
        b0, b1 = TB.bspline(3, 0.0), TB.bspline(3, 1.0)
        np.testing.assert_allclose(y, [b0 * b0, b0 * b0, b0 * b0, b1 * b0], rtol=0, atol=1e-15)


def test_degree0_equals_voxel_path_lengths(orc):
    rng = np.random.default_rng(60)
    dims = (8, 7, 6)
    origin = np.array([0.0, 0.0, 0.0])
    c = rng.uniform(0, 1, size=(6, 7, 8))
    w, s = _random_rays_through(rng, 300, dims, origin)
    g = orc.Geometry("rays", omega=w, s=s)
    ya = orc.forward(0, dims, origin, c, g)
    ys = orc.siddon(dims, origin, c, g)
    assert np.max(np.abs(ya - ys)) <= 1e-12 * max(1.0, np.max(np.abs(ys)))
    # all-ones volume: the path lengths add up to the chord through the box
    ones = np.ones((6, 7, 8))
    y1 = orc.siddon(dims, origin, ones, g)
    ref = np.array([TB.box_chord(origin - 0.5, origin + np.array(dims) - 0.5, s[i], w[i]) for i in range(len(w))])
    np.testing.assert_allclose(y1, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_partition_of_unity_chord(orc, n):
    # c = 1: f = F(x1)F(x2)F(x3) with F = 1 away from the grid border; for a
    # ray whose transverse coordinates stay in that interior, Ac = N_d/|w_d|
    N = 16
    dims = (N, N, N)
    origin = np.zeros(3)
    c = np.ones((N, N, N))
    rng = np.random.default_rng(70 + n)
    ws, ss, ref = [], [], []
    for d in range(3):
        for _ in range(8):
            w = rng.uniform(-0.12, 0.12, 3)
            w[d] = rng.choice([-1.0, 1.0])
            w /= np.linalg.norm(w)
            s = np.full(3, (N - 1) / 2.0) + rng.uniform(-0.5, 0.5, 3)
            ws.append(w)
            ss.append(s)
            ref.append(N / abs(w[d]))
    g = orc.Geometry("rays", omega=np.array(ws), s=np.array(ss))
    y = orc.forward(n, dims, origin, c, g)
    np.testing.assert_allclose(y, ref, rtol=1e-12)


@pytest.mark.parametrize("n", [0, 1, 3])
def test_adjointness(orc, n):
    rng = np.random.default_rng(80 + n)
    dims = (10, 9, 8)
    origin = I.centred_origin(dims)
    c = rng.normal(size=(8, 9, 10))
    geo = I.parallel_views(I.random_directions(rng, 5), 12, 11, 1.0)
    g = orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u,
                     det_v=geo.det_v, nu=geo.nu, nv=geo.nv)
    y = rng.normal(size=g.n_rays)
    Ac = orc.forward(n, dims, origin, c, g)
    ATy = orc.adjoint(n, dims, origin, y, g)
    lhs, rhs = float(Ac @ y), float(np.sum(c * ATy))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) + 1e-12
    # sampled gather form agrees with the scatter form
    k = rng.choice(c.size, 25, replace=False)
    vals, _ = orc.adjoint_at(n, dims, origin, y, g, k)
    np.testing.assert_allclose(vals, ATy.reshape(-1)[k], rtol=1e-12, atol=1e-13)


def _pin_geometries(orc, rng):
    par = I.parallel_views(I.random_directions(rng, 4), 9, 7, 1.0, center=(0.31, -0.2, 0.17))
    cone = I.helical_cone(3, 20.0, 34.0, 11, 8, 1.4, turns=0.7, table_feed=3.0)
    out = []
    for geo in (par, cone):
        kw = dict(det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v, nu=geo.nu, nv=geo.nv)
        if geo.kind == "parallel":
            out.append(orc.Geometry("parallel", direction=geo.src, **kw))
        else:
            out.append(orc.Geometry("cone", source=geo.src, **kw))
    return out


@pytest.mark.parametrize("n", [1, 3])
def test_subset_operators_match_full_operators(orc, n):
    """forward_subset / adjoint_subset (the checkers of the full-size GPU
    tests and of the timed CPU baseline) equal the full operators restricted
    to the same rays: rows of A c, and A^T of a y that is zero off the
    listed rays; pair counts equal count_pairs per ray."""
    rng = np.random.default_rng(140 + n)
    dims = (11, 9, 10)
    origin = I.centred_origin(dims)
    c = rng.normal(size=dims[::-1])
    for g in _pin_geometries(orc, rng):
        rays = np.sort(rng.choice(g.n_rays, 37, replace=False))
        full = orc.forward(n, dims, origin, c, g)
        sub, pairs = orc.forward_subset(n, dims, origin, c, g, rays)
        np.testing.assert_allclose(sub, full[rays], rtol=1e-13, atol=1e-13 * np.abs(full).max())
        _, per = orc.count_pairs(n, dims, origin, g, per_ray=True)
        np.testing.assert_array_equal(pairs, per[rays])
        ys = rng.normal(size=rays.size)
        yfull = np.zeros(g.n_rays)
        yfull[rays] = ys
        ref = orc.adjoint(n, dims, origin, yfull, g)
        got, npair = orc.adjoint_subset(n, dims, origin, ys, g, rays)
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
        assert npair == per[rays].sum()


def test_adjoint_subset_on_a_large_grid(orc):
    """Above 2^24 coefficients adjoint_subset adds into one shared buffer
    with atomic adds instead of per-thread buffers: same sums as the plain
    serial scatter of orc_adjoint (here on a few rays through a 260 x 255 x
    256 grid), and the same as the private-buffer mode on a smaller grid."""
    rng = np.random.default_rng(150)
    dims = (260, 255, 256)
    assert dims[0] * dims[1] * dims[2] > (1 << 24)
    origin = I.centred_origin(dims)
    geo = I.parallel_views(I.random_directions(rng, 2), 3, 2, 37.0)
    g = orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                     nu=geo.nu, nv=geo.nv)
    rays = np.arange(g.n_rays)
    y = rng.uniform(0.5, 1.5, g.n_rays)
    ref = orc.adjoint(3, dims, origin, y, g)
    got, npair = orc.adjoint_subset(3, dims, origin, y, g, rays, nthreads=4)
    nz = np.abs(ref) > 0
    assert nz.sum() > 10000 and npair == orc.count_pairs(3, dims, origin, g)
    assert np.array_equal(np.abs(got) > 0, nz)
    np.testing.assert_allclose(got[nz], ref[nz], rtol=1e-13)


def test_windowed_adjoint_at_matches_adjoint_at(orc):
    """adjoint_at_views (pixel windows of each coefficient's support) gives
    the same values and pair counts as adjoint_at (every ray tested), for
    parallel and cone views, coefficients at corners, faces and inside, and a
    cone whose source sits close enough that some support corners are behind
    its plane (the whole detector is then kept)."""
    rng = np.random.default_rng(160)
    dims = (13, 11, 12)
    origin = I.centred_origin(dims)
    close = I.helical_cone(3, 7.0, 16.0, 15, 13, 1.0, turns=0.5, table_feed=2.0)
    geoms = _pin_geometries(orc, rng) + [orc.Geometry("cone", source=close.src, det_center=close.det_center,
                                                      det_u=close.det_u, det_v=close.det_v, nu=close.nu,
                                                      nv=close.nv)]
    nk = dims[0] * dims[1] * dims[2]
    k = np.unique(np.concatenate([rng.choice(nk, 40, replace=False),
                                  [0, dims[0] - 1, nk - 1, nk // 2, dims[0] * dims[1] * 5 + 6]]))
    for n in (0, 3):
        for g in geoms:
            y = rng.normal(size=g.n_rays)
            ref, pr = orc.adjoint_at(n, dims, origin, y, g, k)
            got, pg = orc.adjoint_at_views(n, dims, origin, y, g, k)
            np.testing.assert_array_equal(pg, pr)
            assert pr.sum() > 0
            np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(ref).max()))


def test_cone_geometry_rays(orc):
    geo = I.helical_cone(3, 100.0, 150.0, 5, 4, 1.5, turns=1.0, table_feed=6.0)
    g = orc.Geometry("cone", source=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                     nu=geo.nu, nv=geo.nv)
    s, w = g.rays()
    for r in range(g.n_rays):
        v, rem = divmod(r, geo.nu * geo.nv)
        iv, iu = divmod(rem, geo.nu)
        q = geo.det_center[v] + (iu - 2.0) * geo.det_u[v] + (iv - 1.5) * geo.det_v[v]
        np.testing.assert_allclose(s[r], geo.src[v], atol=1e-12)
        d = q - geo.src[v]
        np.testing.assert_allclose(w[r], d / np.linalg.norm(d), atol=1e-14)


# --------------------------------------------------------------------------
# pair counts and the Algorithm 2 / 3 enumeration
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 2, 3])
def test_pair_count_matches_brute_force(orc, n):
    rng = np.random.default_rng(90 + n)
    dims = (9, 7, 8)
    origin = np.array([0.5, 0.0, -1.0])
    w, s = _random_rays_through(rng, 40, dims, origin)
    g = orc.Geometry("rays", omega=w, s=s)
    tot, per = orc.count_pairs(n, dims, origin, g, per_ray=True)
    for i in range(len(w)):
        assert per[i] == len(TB.pair_set(n, dims, origin, s[i], w[i]))
    assert tot == per.sum()


@pytest.mark.parametrize("n", [1, 2, 3])
def test_dda_neighbourhood_enumeration(orc, n):
    """Algorithm 2 + 3 with window radius R = n visits every basis whose
    support the ray meets, never twice, with at most three cells per slab;
    R = n + 1 adds only zero contributions; R = n - 1 misses some."""
    rng = np.random.default_rng(100 + n)
    dims = (10, 9, 8)
    origin = np.zeros(3)
    c = rng.normal(size=(8, 9, 10))
    w, s = _random_rays_through(rng, 120, dims, origin, spread=0.6)
    missed_small = 0
    for i in range(len(w)):
        true = TB.pair_set(n, dims, origin, s[i], w[i])
        vis, mc, _ = orc.dda_visit(n, n, dims, origin, s[i], w[i])
        assert len(vis) == len(set(vis.tolist()))
        assert mc <= 3
        assert true <= set(vis.tolist())
        vis1, _, _ = orc.dda_visit(n, n + 1, dims, origin, s[i], w[i])
        assert true <= set(vis1.tolist())
        ctr = lambda k: origin + np.array([k % 10, (k // 10) % 9, k // 90])
        s0 = sum(c.reshape(-1)[k] * orc.footprint(n, w[i], s[i] - ctr(k)) for k in vis)
        s1 = sum(c.reshape(-1)[k] * orc.footprint(n, w[i], s[i] - ctr(k)) for k in vis1)
        assert abs(s0 - s1) <= 1e-13 * max(1.0, abs(s0))
        vis_small, _, _ = orc.dda_visit(n, n - 1, dims, origin, s[i], w[i])
        if not true <= set(vis_small.tolist()):
            missed_small += 1
    assert missed_small > 0


def test_pairs_per_unit_length(orc):
    # expected pairs per unit length = area of the shadow of [-W,W]^3 = (n+1)^2 |w|_1
    n = 3
    N = 40
    dims = (N, N, N)
    origin = I.centred_origin(dims)
    rng = np.random.default_rng(120)
    w = I.random_directions(rng, 400)
    s = rng.uniform(-3, 3, (400, 3))
    g = orc.Geometry("rays", omega=w, s=s)
    _, per = orc.count_pairs(n, dims, origin, g, per_ray=True)
    # length over which bases are enumerated: chord through the grid box of
    # centres dilated by W (exact for these central rays up to the ends)
    L = np.array([TB.box_chord(origin - 2.0, origin + N - 1 + 2.0, s[i], w[i]) for i in range(400)])
    expect = (n + 1) ** 2 * np.abs(w).sum(1) * L
    ratio = per.sum() / expect.sum()
    assert 0.85 < ratio < 1.01


# --------------------------------------------------------------------------
# MLP f_theta (Sec. 2.2) and the loss of Algorithm 1
# --------------------------------------------------------------------------
def _rand_params(orc, sizes, rng, scale=0.5):
    return rng.normal(size=orc.mlp_param_count(sizes)) * scale


def test_mlp_single_unit_logistic(orc):
    # 1 -> 1 -> 1: out = w2 * silu(w1 x + b1) + b2 ; silu(1) = logistic(1)
    sizes = [1, 1, 1]
    prm = np.array([1.0, 0.0, 1.0, 0.0])
    out = orc.mlp_forward(sizes, prm, np.array([[1.0]]))
    assert abs(out[0] - 0.7310585786300049) < 1e-15
    prm = np.array([2.0, -0.5, 3.0, 0.25])  # 3 * silu(2*x - 0.5) + 0.25 at x = 0.75
    out = orc.mlp_forward(sizes, prm, np.array([[0.75]]))
    assert abs(out[0] - (3.0 * 1.0 / (1.0 + math.exp(-1.0)) + 0.25)) < 1e-15


def test_mlp_linear_regime_matches_matrix_product(orc):
    # every pre-activation >= 60: silu(z) = z to double precision, so the
    # network is the affine map W4 (W3 (W2 (W1 x + b1) + b2) + b3) + b4
    sizes = [5, 7, 6, 4, 1]
    rng = np.random.default_rng(130)
    Ws = [rng.uniform(0.1, 1.0, (sizes[i + 1], sizes[i])) for i in range(4)]
    bs = [rng.uniform(60, 70, sizes[i + 1]) for i in range(4)]
    prm = np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in zip(Ws, bs)])
    X = rng.uniform(0, 1, (6, 5))
    out = orc.mlp_forward(sizes, prm, X)
    ref = []
    for x in X:
        h = x
        for W, b in zip(Ws, bs):
            h = W @ h + b
        ref.append(h[0])
    np.testing.assert_allclose(out, ref, rtol=1e-13)


def test_mlp_gradient_finite_differences(orc):
    sizes = [5, 8, 7, 6, 1]
    rng = np.random.default_rng(140)
    prm = _rand_params(orc, sizes, rng)
    X = rng.normal(size=(9, 5))
    Y = rng.normal(size=9)
    L, g = orc.mlp_loss_grad(sizes, prm, X, Y)
    ref_L = np.mean((orc.mlp_forward(sizes, prm, X) - Y) ** 2)
    assert abs(L - ref_L) < 1e-14 * max(1, ref_L)
    eps = 1e-5
    for i in range(len(prm)):
        pp, pm = prm.copy(), prm.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (np.mean((orc.mlp_forward(sizes, pp, X) - Y) ** 2) - np.mean((orc.mlp_forward(sizes, pm, X) - Y) ** 2)) / (
            2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bf16_rounding_ties_to_even(orc):
    assert orc.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert orc.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert orc.bf16_round(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert orc.bf16_round(-3.0) == -3.0
    assert orc.bf16_round(0.1) == 0.10009765625


def test_mlp_bf16_contract_changes_little(orc):
    sizes = [5, 64, 64, 64, 1]
    rng = np.random.default_rng(150)
    prm = _rand_params(orc, sizes, rng, scale=0.15)
    X = rng.uniform(-1, 1, (50, 5))
    a = orc.mlp_forward(sizes, prm, X, mode=0)
    b = orc.mlp_forward(sizes, prm, X, mode=1)
    c2 = orc.mlp_forward(sizes, prm, X, mode=2)
    assert 0 < np.max(np.abs(a - b)) < 0.05 * np.max(np.abs(a))
    # split activations remove most of the activation-rounding error
    assert np.max(np.abs(c2 - b)) > 0


def test_features_invariance_and_frame(orc):
    rng = np.random.default_rng(160)
    for n in (2, 3):
        W = 0.5 * (n + 1)
        for _ in range(50):
            w = rng.normal(size=3)
            w /= np.linalg.norm(w)
            p = rng.uniform(-2, 2, 3)
            f = orc.features(n, w, p)
            # canonical direction in the chamber 0 <= w1 <= w2 <= w3
            assert 0 <= f[0] <= f[1] <= f[2]
            np.testing.assert_allclose(np.sort(np.abs(w)), f[:3], atol=1e-15)
            # (u, v) components carry the projection of p on H_w
            pp = p - (p @ w) * w
            assert abs((f[3] ** 2 + f[4] ** 2) * (W * W / 3.0) - pp @ pp) < 1e-12
            # invariant along w and under signed permutations
            np.testing.assert_allclose(orc.features(n, w, p + 3.3 * w), f, atol=1e-13)
            perm = rng.permutation(3)
            sg = rng.choice([-1.0, 1.0], 3)
            np.testing.assert_allclose(orc.features(n, sg * w[perm], sg * p[perm]), f, atol=1e-13)


def test_forward_mlp_constant_network_counts_pairs(orc):
    sizes = [5, 4, 3, 1]
    prm = np.zeros(orc.mlp_param_count(sizes))
    prm[-1] = 0.75  # output bias
    dims = (6, 7, 5)
    origin = I.centred_origin(dims)
    rng = np.random.default_rng(170)
    w, s = _random_rays_through(rng, 30, dims, origin)
    g = orc.Geometry("rays", omega=w, s=s)
    y = orc.forward_mlp(3, dims, origin, np.ones((5, 7, 6)), g, sizes, prm, mode=0)
    _, per = orc.count_pairs(3, dims, origin, g, per_ray=True)
    np.testing.assert_allclose(y, 0.75 * per, rtol=1e-14)


# --------------------------------------------------------------------------
# input generators that both sides consume
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_prefilter_interpolates_samples(orc, n):
    rng = np.random.default_rng(180)
    s = rng.uniform(0, 1, (5, 6, 7))
    c = I.prefilter(s, n)
    X = np.stack(np.meshgrid(np.arange(7), np.arange(6), np.arange(5), indexing="xy"), -1)
    # points in C-order [z][y][x]
    pts = np.array([[x, y, z] for z in range(5) for y in range(6) for x in range(7)], dtype=float)
    vals = TB.spline_on_points(n, c, np.zeros(3), pts)
    np.testing.assert_allclose(vals, s.reshape(-1), atol=1e-12)
    del X


def test_ellipsoid_line_integral_sphere_chord():
    ell = I.Ellipsoids(np.array([[1.0, -2.0, 0.5]]), np.array([[3.0, 3.0, 3.0]]), np.eye(3)[None], np.array([0.7]))
    s = np.array([[1.0, -2.0, -40.0], [2.5, -2.0, 0.0], [1.0, 5.0, 0.5]])
    w = np.array([[0, 0, 1.0], [0, 1.0, 0], [1.0, 0, 0]])
    y = I.ellipsoid_line_integrals(ell, s, w)
    # second ray: distance to the centre sqrt(1.5^2 + 0.5^2)
    np.testing.assert_allclose(y, [0.7 * 6.0, 0.7 * 2 * math.sqrt(9 - 1.5 ** 2 - 0.5 ** 2), 0.0], atol=1e-12)
