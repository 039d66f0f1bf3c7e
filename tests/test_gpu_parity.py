"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Element-by-element comparisons on seeded inputs at sizes the oracle finishes
in seconds (several 16x8 detector tiles and 16^3 coefficient bricks with
ragged tails), plus sampled comparisons at the full size of the 128^3
tilt-series workload in the launch configuration the benchmark times.
Tolerance: relative L2 error <= 1e-5 for FP32 forward and adjoint against
the FP64 oracle (the target the method is held to); footprints within
2e-6 of the footprint peak (FP32 node arithmetic).
"""
import numpy as np
import pytest

from paper_2511_11078_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import spl

    B.build()
    spl.lib()
    assert torch.cuda.is_available()
    return torch, spl


def oracle_geom(orc, geo):
    if geo.kind == "rays":
        return orc.Geometry("rays", omega=geo.omega, s=geo.s)
    if geo.kind == "parallel":
        return orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u,
                            det_v=geo.det_v, nu=geo.nu, nv=geo.nv)
    return orc.Geometry("cone", source=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                        nu=geo.nu, nv=geo.nv)


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_forward(env, dims, origin, geo, c, degree, kahan=True):
    torch, spl = env
    g = spl.Geometry(dims, origin, geo)
    ct = torch.tensor(np.asarray(c, dtype=np.float32), device="cuda")
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    spl.forward(g, ct, y, spl.basis(degree, kahan=kahan))
    g.status()
    return y.cpu().numpy().astype(np.float64)


def gpu_adjoint(env, dims, origin, geo, y, degree, form=0):
    torch, spl = env
    g = spl.Geometry(dims, origin, geo)
    yt = torch.tensor(np.asarray(y, dtype=np.float32), device="cuda")
    c = torch.full(g.coeff_shape, float("nan"), dtype=torch.float32, device="cuda")
    spl.adjoint(g, yt, c, spl.basis(degree, adjoint=form))
    g.status()
    return c.cpu().numpy().astype(np.float64)


DIMS = (20, 18, 17)  # two 16-bricks per axis with ragged tails


def parallel_geometry(rng, nu=21, nv=19, shift=(0.137, -0.271, 0.093)):
    dirs = np.concatenate([
        I.random_directions(rng, 4),
        np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 0, 1.0],
                  [np.cos(0.5), np.sin(0.5), 0.0],
                  [1.0, 1.0, 1.0], [1.0, -1.0, 0.0], [-1.0, 1.0, 1.0]]),
    ])
    return I.parallel_views(dirs, nu, nv, 1.0, center=shift)


def cone_geometry(nu=23, nv=17):
    return I.helical_cone(4, 60.0, 90.0, nu, nv, 1.3, turns=0.8, table_feed=5.0)


def ray_geometry(rng, dims, origin):
    w = I.random_directions(rng, 150)
    ctr = origin + (np.asarray(dims) - 1) / 2.0
    s = ctr + rng.uniform(-8, 8, (150, 3)) + rng.uniform(-30, 30, (150, 1)) * w
    extra_w = np.array([[0, 0, 1.0], [0, 1.0, 0], [1.0, 0, 0], [1, 1, 0.0], [1, 1, 1.0], [0, 1, -1.0], [1e-9, 0, 1.0]])
    extra_s = ctr + np.array([[0.3, 0.2, 0], [1.1, 0, -0.4], [0, 2.5, 1.5], [0, 0, 0.7], [0.2, -0.1, 0.3],
                              [-3.0, 0.4, 0.4], [0.5, 0.5, 0]])
    # rays that miss the volume entirely
    miss_w = np.array([[0, 0, 1.0], [1.0, 0, 0]])
    miss_s = ctr + np.array([[40.0, 0, 0], [0, 0, 35.0]])
    return I.RayGeometry(np.concatenate([w, extra_w, miss_w]), np.concatenate([s, extra_s, miss_s]))


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_forward_parallel(env, orc, degree):
    rng = np.random.default_rng(1000 + degree)
    origin = I.centred_origin(DIMS)
    c = rng.normal(size=DIMS[::-1]).astype(np.float32).astype(np.float64)
    geo = parallel_geometry(rng)
    y = gpu_forward(env, DIMS, origin, geo, c, degree)
    yref = orc.forward(degree, DIMS, origin, c, oracle_geom(orc, geo))
    assert rel_l2(y, yref) <= TOL, rel_l2(y, yref)
    assert np.max(np.abs(y - yref)) <= 1e-4 * np.max(np.abs(yref))


@pytest.mark.parametrize("degree", [1, 3])
def test_forward_cone(env, orc, degree):
    rng = np.random.default_rng(1100 + degree)
    origin = I.centred_origin(DIMS)
    c = rng.uniform(0, 1, size=DIMS[::-1]).astype(np.float32).astype(np.float64)
    geo = cone_geometry()
    y = gpu_forward(env, DIMS, origin, geo, c, degree)
    yref = orc.forward(degree, DIMS, origin, c, oracle_geom(orc, geo))
    assert rel_l2(y, yref) <= TOL, rel_l2(y, yref)


@pytest.mark.parametrize("degree", [0, 2, 3])
def test_forward_explicit_rays(env, orc, degree):
    rng = np.random.default_rng(1200 + degree)
    origin = I.centred_origin(DIMS) + np.array([0.25, -0.5, 3.0])
    c = rng.normal(size=DIMS[::-1]).astype(np.float32).astype(np.float64)
    geo = ray_geometry(rng, DIMS, origin)
    y = gpu_forward(env, DIMS, origin, geo, c, degree)
    yref = orc.forward(degree, DIMS, origin, c, oracle_geom(orc, geo))
    assert rel_l2(y, yref) <= TOL, rel_l2(y, yref)
    assert y[-1] == 0.0 and y[-2] == 0.0  # rays that miss the grid


@pytest.mark.parametrize("kind", ["parallel", "cone", "rays"])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_forward_direct(env, orc, kind, degree):
    """SPL_FP_DIRECT: the forward as the line integral of f itself (same
    pieces and nodes, a window of coefficients) against the oracle, and
    adjoint to the footprint-form A^T."""
    torch, spl = env
    rng = np.random.default_rng(1250 + degree)
    origin = I.centred_origin(DIMS)
    geo = {"parallel": parallel_geometry(rng), "cone": cone_geometry(),
           "rays": ray_geometry(rng, DIMS, origin)}[kind]
    c = rng.normal(size=DIMS[::-1]).astype(np.float32)
    g = spl.Geometry(DIMS, origin, geo)
    ct = torch.tensor(c, device="cuda")
    y = torch.full((g.n_rays,), float("nan"), dtype=torch.float32, device="cuda")
    spl.forward(g, ct, y, spl.basis(degree, spl.SPL_FP_DIRECT))
    g.status()
    got = y.cpu().numpy().astype(np.float64)
    yref = orc.forward(degree, DIMS, origin, c.astype(np.float64), oracle_geom(orc, geo))
    assert np.all(np.isfinite(got))
    assert rel_l2(got, yref) <= TOL, rel_l2(got, yref)
    yy = rng.normal(size=g.n_rays).astype(np.float32)
    ca = torch.empty(g.coeff_shape, dtype=torch.float32, device="cuda")
    spl.adjoint(g, torch.tensor(yy, device="cuda"), ca, spl.basis(degree, spl.SPL_FP_DIRECT))
    g.status()
    lhs = float(got @ yy.astype(np.float64))
    rhs = float(np.sum(c.astype(np.float64) * ca.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(got) * np.linalg.norm(yy), (lhs, rhs)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_adjoint_parallel(env, orc, degree, form):
    rng = np.random.default_rng(1300 + degree)
    origin = I.centred_origin(DIMS)
    geo = parallel_geometry(rng)
    y = rng.normal(size=geo.n_rays).astype(np.float32).astype(np.float64)
    c = gpu_adjoint(env, DIMS, origin, geo, y, degree, form)
    cref = orc.adjoint(degree, DIMS, origin, y, oracle_geom(orc, geo))
    assert np.all(np.isfinite(c))
    assert rel_l2(c, cref) <= TOL, rel_l2(c, cref)


@pytest.mark.parametrize("degree", [1, 3])
def test_adjoint_cone(env, orc, degree):
    rng = np.random.default_rng(1400 + degree)
    origin = I.centred_origin(DIMS)
    geo = cone_geometry()
    y = rng.uniform(-1, 1, size=geo.n_rays).astype(np.float32).astype(np.float64)
    c = gpu_adjoint(env, DIMS, origin, geo, y, degree)
    cref = orc.adjoint(degree, DIMS, origin, y, oracle_geom(orc, geo))
    assert rel_l2(c, cref) <= TOL, rel_l2(c, cref)


@pytest.mark.parametrize("degree", [0, 3])
def test_adjoint_explicit_rays(env, orc, degree):
    rng = np.random.default_rng(1500 + degree)
    origin = I.centred_origin(DIMS)
    geo = ray_geometry(rng, DIMS, origin)
    y = rng.normal(size=geo.n_rays).astype(np.float32).astype(np.float64)
    c = gpu_adjoint(env, DIMS, origin, geo, y, degree)
    cref = orc.adjoint(degree, DIMS, origin, y, oracle_geom(orc, geo))
    assert rel_l2(c, cref) <= TOL, rel_l2(c, cref)


def b_axis_rays(rng, dims, origin, axis, count):
    """Rays whose smallest direction component is along `axis` (the b axis
    the scatter adjoint keeps contiguous), with both signs of every
    component, through the middle of the grid."""
    w = rng.normal(size=(count, 3))
    w[:, axis] *= 0.15
    w *= np.where(rng.uniform(size=(count, 3)) < 0.5, -1.0, 1.0)
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    ctr = origin + (np.asarray(dims) - 1) / 2.0
    s = ctr + rng.uniform(-5, 5, (count, 3))
    return w, s


@pytest.mark.parametrize("axis", [0, 1, 2, -1])
def test_adjoint_layout_per_b_axis(env, orc, axis):
    """The scatter adjoint reduces each ray into the layout of c whose
    contiguous axis is the ray's b axis (x, y or z fast, four shifted copies
    each) and folds the layouts back: rays of each b axis alone, and all
    three mixed (axis -1), on a grid whose sizes are not multiples of 4."""
    rng = np.random.default_rng(2600 + axis)
    dims = (19, 22, 13)
    origin = I.centred_origin(dims)
    axes = [axis] if axis >= 0 else [0, 1, 2]
    parts = [b_axis_rays(rng, dims, origin, a, 120) for a in axes]
    geo = I.RayGeometry(np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
    y = rng.normal(size=geo.n_rays).astype(np.float32).astype(np.float64)
    c = gpu_adjoint(env, dims, origin, geo, y, 3)
    cref = orc.adjoint(3, dims, origin, y, oracle_geom(orc, geo))
    assert np.isfinite(c).all()
    assert rel_l2(c, cref) <= TOL, rel_l2(c, cref)


@pytest.mark.parametrize("kind", ["parallel", "cone"])
@pytest.mark.parametrize("degree", [1, 3])
def test_adjoint_scatter_form(env, orc, kind, degree):
    """The ray-driven scatter form of A^T gives the same result as the
    gather form and the oracle."""
    torch, spl = env
    rng = np.random.default_rng(1550 + degree)
    origin = I.centred_origin(DIMS)
    geo = parallel_geometry(rng) if kind == "parallel" else cone_geometry()
    y = rng.normal(size=geo.n_rays).astype(np.float32)
    g = spl.Geometry(DIMS, origin, geo)
    yt = torch.tensor(y, device="cuda")
    cs = torch.full(g.coeff_shape, float("nan"), dtype=torch.float32, device="cuda")
    cgat = torch.empty_like(cs)
    spl.adjoint(g, yt, cs, spl.basis(degree, adjoint=spl.SPL_ADJ_SCATTER))
    spl.adjoint(g, yt, cgat, spl.basis(degree, adjoint=spl.SPL_ADJ_GATHER))
    g.status()
    cref = orc.adjoint(degree, DIMS, origin, y.astype(np.float64), oracle_geom(orc, geo))
    a = cs.cpu().numpy().astype(np.float64)
    b = cgat.cpu().numpy().astype(np.float64)
    assert rel_l2(a, cref) <= TOL and rel_l2(b, cref) <= TOL
    assert rel_l2(a, b) <= 1e-6


def tilt_geometry(axis, n_views=7, nu=37, nv=21, center=(0.21, -0.37, 0.44)):
    """Single-axis tilt about coordinate axis `axis` (slice-separable views:
    flat directions, detector rows along the axis), plus views that are not
    separable: a flat direction with a rolled detector, a second tilt group
    whose detector centre sits at another height, and a general direction."""
    e = np.eye(3)
    b = e[axis]
    p, q = [e[i] for i in range(3) if i != axis]
    t = np.pi * (np.arange(n_views) + 0.3) / n_views
    d = np.cos(t)[:, None] * p + np.sin(t)[:, None] * q
    du = np.cross(b, d)
    dv = np.tile(b, (n_views, 1))
    dc = np.tile(np.asarray(center, dtype=np.float64), (n_views, 1))
    w = np.cos(0.7) * p + np.sin(0.7) * q
    u0 = np.cross(b, w)
    phi = 0.3
    roll_u, roll_v = np.cos(phi) * u0 + np.sin(phi) * b, -np.sin(phi) * u0 + np.cos(phi) * b
    w2 = np.cos(1.9) * p + np.sin(1.9) * q
    g = np.array([0.3, 0.5, 0.8]) / np.linalg.norm([0.3, 0.5, 0.8])
    gu, gv = I.detector_frame(g)
    src = np.concatenate([d, [w, w2, g]])
    dcs = np.concatenate([dc, [center, np.asarray(center) + 0.5 * b, center]])
    dus = np.concatenate([du, [roll_u, np.cross(b, w2), gu]])
    dvs = np.concatenate([dv, [roll_v, b, gv]])
    return I.ViewGeometry("parallel", src, dcs, dus, dvs, nu, nv)


@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_separable_views(env, orc, axis, degree):
    """Slice-separable views through the plane matrices (SPL_SEP_AUTO) and
    walked ray by ray (SPL_SEP_OFF): forward and adjoint against the oracle,
    every output written, and <A c, y> = <c, A^T y> for the plane path."""
    torch, spl = env
    rng = np.random.default_rng(1560 + 10 * axis + degree)
    origin = I.centred_origin(DIMS)
    geo = tilt_geometry(axis)
    g = spl.Geometry(DIMS, origin, geo)
    c = rng.normal(size=DIMS[::-1]).astype(np.float32)
    y = rng.normal(size=geo.n_rays).astype(np.float32)
    ct, yt = torch.tensor(c, device="cuda"), torch.tensor(y, device="cuda")
    og = oracle_geom(orc, geo)
    yref = orc.forward(degree, DIMS, origin, c.astype(np.float64), og)
    cref = orc.adjoint(degree, DIMS, origin, y.astype(np.float64), og)
    out = {}
    for sep in (spl.SPL_SEP_AUTO, spl.SPL_SEP_OFF):
        for form in (spl.SPL_ADJ_SCATTER, spl.SPL_ADJ_GATHER):
            bas = spl.basis(degree, separable=sep, adjoint=form)
            yo = torch.full((g.n_rays,), float("nan"), dtype=torch.float32, device="cuda")
            co = torch.full(g.coeff_shape, float("nan"), dtype=torch.float32, device="cuda")
            spl.forward(g, ct, yo, bas)
            spl.adjoint(g, yt, co, bas)
            g.status()
            yo = yo.cpu().numpy().astype(np.float64)
            co = co.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(yo)) and np.all(np.isfinite(co))
            assert rel_l2(yo, yref) <= TOL, (sep, form, rel_l2(yo, yref))
            assert rel_l2(co, cref) <= TOL, (sep, form, rel_l2(co, cref))
            out[sep, form] = (yo, co)
    ya, ca = out[spl.SPL_SEP_AUTO, spl.SPL_ADJ_SCATTER]
    lhs = float(ya @ y.astype(np.float64))
    rhs = float(np.sum(c.astype(np.float64) * ca))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(ya) * np.linalg.norm(y), (lhs, rhs)


def test_separable_tall_detector(env, orc):
    """More detector rows than one pass of the row gather covers (nv > 256),
    most of them above or below the grid."""
    torch, spl = env
    rng = np.random.default_rng(1590)
    dims = (12, 10, 9)
    origin = I.centred_origin(dims)
    geo = I.tilt_series(5, 15, 300, 0.11)
    c = rng.normal(size=dims[::-1]).astype(np.float32).astype(np.float64)
    y = gpu_forward(env, dims, origin, geo, c, 3)
    yref = orc.forward(3, dims, origin, c, oracle_geom(orc, geo))
    assert rel_l2(y, yref) <= TOL, rel_l2(y, yref)
    yy = rng.normal(size=geo.n_rays).astype(np.float32).astype(np.float64)
    ca = gpu_adjoint(env, dims, origin, geo, yy, 3)
    cref = orc.adjoint(3, dims, origin, yy, oracle_geom(orc, geo))
    assert rel_l2(ca, cref) <= TOL, rel_l2(ca, cref)


@pytest.mark.parametrize("kind", ["parallel", "cone", "rays"])
def test_dot_product_adjointness(env, kind):
    """<A c, y> = <c, A^T y> for the GPU operators (FP32 arithmetic, FP64
    inner products of the outputs)."""
    rng = np.random.default_rng(1600)
    origin = I.centred_origin(DIMS)
    geo = {"parallel": parallel_geometry(rng), "cone": cone_geometry(), "rays": ray_geometry(rng, DIMS, origin)}[kind]
    c = rng.normal(size=DIMS[::-1]).astype(np.float32)
    y = rng.normal(size=geo.n_rays).astype(np.float32)
    Ac = gpu_forward(env, DIMS, origin, geo, c, 3)
    ATy = gpu_adjoint(env, DIMS, origin, geo, y, 3)
    lhs = float(Ac @ y.astype(np.float64))
    rhs = float(np.sum(c.astype(np.float64) * ATy))
    scale = np.linalg.norm(Ac) * np.linalg.norm(y)
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs)


def test_axis_aligned_rays_on_voxel_faces(env, orc):
    """Degree 0 with rays lying in voxel faces (half-open cells): same
    convention as the oracle."""
    dims = (6, 5, 4)
    origin = np.zeros(3)
    rng = np.random.default_rng(1700)
    c = rng.uniform(0, 1, size=(4, 5, 6)).astype(np.float32).astype(np.float64)
    w = np.array([[0, 0, 1.0], [0, 1.0, 0], [1.0, 0, 0], [0, 0, 1.0]])
    s = np.array([[2.5, 1.5, 0.0], [0.5, 0.0, 1.5], [0.0, 3.5, 2.5], [-0.5, 1.0, 0]])
    geo = I.RayGeometry(w, s)
    y = gpu_forward(env, dims, origin, geo, c, 0)
    yref = orc.forward(0, dims, origin, c, oracle_geom(orc, geo))
    np.testing.assert_allclose(y, yref, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_footprint_exact(env, orc, degree):
    torch, spl = env
    rng = np.random.default_rng(1800 + degree)
    w, p = I.footprint_samples(rng, 4096, degree)
    p = p + rng.uniform(-3, 3, (4096, 1)) * w  # shift along the line
    w32 = w.astype(np.float32)
    p32 = p.astype(np.float32)
    out = torch.empty(4096, dtype=torch.float32, device="cuda")
    spl.footprint(spl.basis(degree), torch.tensor(w32, device="cuda"), torch.tensor(p32, device="cuda"), out)
    ref = orc.footprint_batch(degree, w32.astype(np.float64), p32.astype(np.float64))
    err = np.max(np.abs(out.cpu().numpy() - ref))
    assert err <= 2e-6 * ref.max(), err


@pytest.mark.parametrize("degree", [0, 3])
def test_pair_count(env, orc, degree):
    """The contribution count (the metric's denominator) is index work: the
    GPU count equals the oracle's, ray by ray, on parallel, tilt (a zero
    direction component), cone and explicit-ray geometries."""
    torch, spl = env
    rng = np.random.default_rng(1900 + degree)
    origin = I.centred_origin(DIMS)
    for geo in (parallel_geometry(rng), tilt_geometry(0), cone_geometry(), ray_geometry(rng, DIMS, origin)):
        g = spl.Geometry(DIMS, origin, geo)
        per, tot = spl.count_pairs_per_ray(g, degree)
        g.status()
        ref_tot, ref = orc.count_pairs(degree, DIMS, origin, oracle_geom(orc, geo), per_ray=True)
        assert tot == ref_tot, (geo.kind, tot, ref_tot)
        np.testing.assert_array_equal(per.cpu().numpy().astype(np.int64), ref)
        assert spl.count_pairs(g, degree) == ref_tot


def grazing_rays(dims, origin, n):
    """Rays that touch support boundaries: axis-aligned and diagonal lines
    whose transverse coordinates sit exactly on, or one ulp beside, the
    faces k +- W of a basis support, lines along support edges, lines
    through support corners, and lines lying in knot planes."""
    W = 0.5 * (n + 1)
    org = np.asarray(origin)
    ctr = org + (np.asarray(dims) - 1) // 2
    w, s = [], []
    for off in (W, -W, np.nextafter(W, 0), np.nextafter(W, 10), 0.5, 1.0, 0.0):
        for ax in range(3):
            d = np.zeros(3)
            d[ax] = 1.0
            t = [(ax + 1) % 3, (ax + 2) % 3]
            p = ctr.copy()
            p[t[0]] += off
            w.append(d.copy())
            s.append(p.copy())
            p[t[1]] += off  # along a support edge
            w.append(d.copy())
            s.append(p.copy())
    for v in ([1, 1, 0], [1, 1, 1], [1, -1, 1], [0, 1, 1], [1, 2, 0]):
        d = np.asarray(v, dtype=np.float64)
        for off in (W, np.nextafter(W, 0), 0.0):
            p = ctr + np.array([off, 0.0, 0.0])  # passes through support corners / edges
            w.append(d.copy())
            s.append(p)
    return I.RayGeometry(np.array(w), np.array(s))


@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_pair_count_grazing_and_face_rays(env, orc, degree):
    torch, spl = env
    origin = I.centred_origin(DIMS)
    geo = grazing_rays(DIMS, origin, degree)
    g = spl.Geometry(DIMS, origin, geo)
    per, tot = spl.count_pairs_per_ray(g, degree)
    g.status()
    ref_tot, ref = orc.count_pairs(degree, DIMS, origin, oracle_geom(orc, geo), per_ray=True)
    np.testing.assert_array_equal(per.cpu().numpy().astype(np.int64), ref)
    assert tot == ref_tot


def test_kahan_off_still_accurate(env, orc):
    rng = np.random.default_rng(2000)
    origin = I.centred_origin(DIMS)
    c = rng.uniform(0, 1, size=DIMS[::-1]).astype(np.float32).astype(np.float64)
    geo = parallel_geometry(rng)
    yref = orc.forward(3, DIMS, origin, c, oracle_geom(orc, geo))
    y0 = gpu_forward(env, DIMS, origin, geo, c, 3, kahan=False)
    y1 = gpu_forward(env, DIMS, origin, geo, c, 3, kahan=True)
    assert rel_l2(y0, yref) <= TOL and rel_l2(y1, yref) <= TOL


def test_empty_and_single_coefficient_grids(env, orc):
    torch, spl = env
    # a grid of one coefficient: A c is the footprint of that basis
    dims = (1, 1, 1)
    origin = np.array([0.2, -0.1, 0.3])
    rng = np.random.default_rng(2100)
    geo = ray_geometry(rng, dims, origin)
    c = np.array([[[1.5]]])
    y = gpu_forward(env, dims, origin, geo, c, 3)
    yref = orc.forward(3, dims, origin, c, oracle_geom(orc, geo))
    assert rel_l2(y, yref) <= TOL
    # a geometry with no views: launches nothing, succeeds
    g = spl.Geometry((4, 4, 4), np.zeros(3), I.ViewGeometry("parallel", np.zeros((0, 3)), np.zeros((0, 3)),
                                                            np.zeros((0, 3)), np.zeros((0, 3)), 4, 4))
    assert g.n_rays == 0
    yt = torch.empty(0, dtype=torch.float32, device="cuda")
    ct = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    spl.forward(g, ct, yt, spl.basis(3))
    spl.adjoint(g, yt, ct, spl.basis(3))
    torch.cuda.synchronize()
    assert float(ct.abs().sum()) == 0.0


def test_stepcap_flag_reports_error(env):
    """Lower the per-slab loop bound: kernels stop early (bounded loops, no
    hang), set the geometry's error flag, and the status call reports it."""
    torch, spl = env
    rng = np.random.default_rng(2200)
    origin = I.centred_origin(DIMS)
    geo = parallel_geometry(rng)
    g = spl.Geometry(DIMS, origin, geo)
    ct = torch.ones(DIMS[::-1], dtype=torch.float32, device="cuda")
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    L = spl.lib()
    old = L.spl_debug_set_iter_cap(2)
    try:
        spl.forward(g, ct, y, spl.basis(3))
        with pytest.raises(spl.SplError) as ei:
            g.status()
        assert ei.value.status == 4
    finally:
        L.spl_debug_set_iter_cap(old)
    spl.forward(g, ct, y, spl.basis(3))
    g.status()  # flag was cleared, normal bound restored


def test_dot_f64_and_cg_steps(env):
    torch, spl = env
    rng = np.random.default_rng(2300)
    work = spl.dot_workspace()
    for n in (0, 1, 7, 1000003):
        a = rng.normal(size=n).astype(np.float32)
        b = rng.normal(size=n).astype(np.float32)
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        at, bt = torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda")
        spl.dot_f64(at, bt, out, work)
        v1 = float(out.item())
        spl.dot_f64(at, bt, out, work)
        assert float(out.item()) == v1  # deterministic
        ref = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        assert abs(v1 - ref) <= 1e-12 * max(1.0, np.sum(np.abs(a.astype(np.float64) * b)))
    n, m = 1000, 777
    x = rng.normal(size=n).astype(np.float32)
    p = rng.normal(size=n).astype(np.float32)
    r = rng.normal(size=m).astype(np.float32)
    q = rng.normal(size=m).astype(np.float32)
    T = lambda v: torch.tensor(v, device="cuda")
    xt, pt, rt, qt = T(x), T(p), T(r), T(q)
    num = torch.tensor([3.0], dtype=torch.float64, device="cuda")
    den = torch.tensor([4.0], dtype=torch.float64, device="cuda")
    spl.cg_step_x(xt, pt, rt, qt, num, den)
    np.testing.assert_allclose(xt.cpu().numpy(), x + 0.75 * p, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(rt.cpu().numpy(), r - 0.75 * q, rtol=1e-6, atol=1e-6)
    st = T(q[:n] if m >= n else rng.normal(size=n).astype(np.float32))
    spl.cg_step_p(pt, st, num, den)
    np.testing.assert_allclose(pt.cpu().numpy(), st.cpu().numpy() + 0.75 * p, rtol=1e-6, atol=1e-6)


# ---------------------------------------------------------------- full size, sampled
# At the benchmark's sizes and launch configuration (the whole geometry in
# one call), against the oracle on dense seeded samples: >= 4096 rays per
# view class (slice-separable tilt views, general parallel views, circular
# cone, helical cone), stratified to include detector edge rows and columns,
# the detector centre and the first and last views (ray ends, rays through
# the truncated volume corners of the cone workloads), and >= 512
# coefficients of A^T, stratified to include the grid's corners, edges and
# faces.
N_RAYS = 4096
N_COEFFS = 512


def stratified_rays(geo, views, count, seed):
    """`count` rays of the listed views: 7/8 uniform, the rest on detector
    edges, the centre and the first and last of the views."""
    rng = np.random.default_rng(seed)
    views = np.asarray(views)
    per = geo.nu * geo.nv
    k_extra = count // 8
    v = views[rng.integers(0, views.size, count)]
    iu = rng.integers(0, geo.nu, count)
    iv = rng.integers(0, geo.nv, count)
    which = rng.integers(0, 6, k_extra)
    e = slice(count - k_extra, count)
    iu[e] = np.where(which == 0, 0, np.where(which == 1, geo.nu - 1, iu[e]))
    iv[e] = np.where(which == 2, 0, np.where(which == 3, geo.nv - 1, iv[e]))
    iu[e] = np.where(which == 4, geo.nu // 2, iu[e])
    iv[e] = np.where(which == 4, geo.nv // 2, iv[e])
    v[e] = np.where(which == 5, views[0], v[e])
    v[count - k_extra:count - k_extra + k_extra // 6] = views[-1]
    return np.unique((v.astype(np.int64) * geo.nv + iv) * geo.nu + iu)


def stratified_coeffs(dims, count, seed):
    """`count` coefficients: 3/4 uniform, the rest on the grid's corners,
    edges and faces."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    k = rng.integers(0, [nx, ny, nz], size=(count, 3))
    m = count // 4
    for r in range(count - m, count):
        for d, nd in enumerate((nx, ny, nz)):
            if rng.uniform() < 0.6:
                k[r, d] = rng.choice([0, 1, nd - 2, nd - 1])
    return np.unique((k[:, 2].astype(np.int64) * ny + k[:, 1]) * nx + k[:, 0])


def full_size_check(env, orc, wl, class_views, seed):
    """Forward and adjoint of the whole workload geometry on the GPU; the
    rays of each view class and the sampled coefficients against the
    oracle."""
    torch, spl = env
    geo = wl.geometry
    g = spl.Geometry(wl.dims, wl.origin, geo)
    og = oracle_geom(orc, geo)
    c64 = wl.coeffs.astype(np.float64)
    ct = torch.tensor(wl.coeffs, device="cuda")
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    spl.forward(g, ct, y, spl.basis(3))
    g.status()
    yh = y.cpu().numpy().astype(np.float64)
    per, _ = spl.count_pairs_per_ray(g, 3)
    g.status()
    per = per.cpu().numpy().astype(np.int64)
    for name, views in class_views.items():
        rays = stratified_rays(geo, views, N_RAYS, seed)
        assert rays.size >= N_RAYS * 0.97
        yref, pairs = orc.forward_subset(3, wl.dims, wl.origin, c64, og, rays)
        assert pairs.sum() > 0, name
        err = rel_l2(yh[rays], yref)
        assert err <= TOL, (name, err)
        # the contribution count of every sampled ray, exactly
        np.testing.assert_array_equal(per[rays], pairs)
    # mixed signs, as a CG residual: the hard case for the adjoint's sums
    rng = np.random.default_rng(seed + 1)
    yv = rng.normal(size=g.n_rays).astype(np.float32)
    cb = torch.full(g.coeff_shape, float("nan"), dtype=torch.float32, device="cuda")
    spl.adjoint(g, torch.tensor(yv, device="cuda"), cb, spl.basis(3))
    g.status()
    k = stratified_coeffs(wl.dims, N_COEFFS + 40, seed + 2)
    assert k.size >= N_COEFFS
    ref, npair = orc.adjoint_at_views(3, wl.dims, wl.origin, yv.astype(np.float64), og, k)
    got = cb.cpu().numpy().reshape(-1)[k].astype(np.float64)
    assert np.isfinite(got).all() and npair.sum() > 0
    err = rel_l2(got, ref)
    assert err <= TOL, err


def test_full_size_tilt128(env, orc):
    """128^3 cubic, 244 parallel views of 192x192: the 180 slice-separable
    tilt views (plane matrices) and the 64 general views (piece march); the
    whole workload's contribution count equals the oracle's."""
    torch, spl = env
    wl = I.workload_tilt(3)
    src = np.asarray(wl.geometry.src)
    flat = np.nonzero(np.any(src == 0.0, axis=1))[0]
    gen = np.nonzero(~np.any(src == 0.0, axis=1))[0]
    full_size_check(env, orc, wl, {"separable": flat, "general": gen}, 2400)
    g = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    assert spl.count_pairs(g, 3) == orc.count_pairs(3, wl.dims, wl.origin, oracle_geom(orc, wl.geometry))


def test_full_size_cone256(env, orc):
    """256^3 cubic, circular cone beam, 360 views of 384x384 (the detector
    truncates the volume corners)."""
    wl = I.workload_cone()
    full_size_check(env, orc, wl, {"cone": np.arange(wl.geometry.n_views)}, 2600)


def test_full_size_helical512(env, orc):
    """512^3 cubic, helical cone beam, 720 views of 768x768: the benchmark's
    headline workload in its launch configuration."""
    wl = I.workload_helical()
    full_size_check(env, orc, wl, {"helical": np.arange(wl.geometry.n_views)}, 2700)


@pytest.mark.parametrize("kind", ["cone", "parallel"])
def test_adjoint_batched_over_views(env, orc, kind):
    """Geometries with more than 48 views scatter the adjoint in batches of
    views (FP32 atomics) added in an FP64 total: the result matches the
    oracle, for cone views and for parallel views with separable,
    flat and general classes (the plane path's part joins the total)."""
    torch, spl = env
    rng = np.random.default_rng(1200)
    dims = (14, 13, 12)
    origin = I.centred_origin(dims)
    if kind == "cone":
        geo = I.helical_cone(101, 40.0, 70.0, 9, 8, 2.2, turns=1.3, table_feed=4.0)
    else:
        t = tilt_geometry(2, n_views=40, nu=13, nv=11)
        extra = I.parallel_views(I.random_directions(rng, 70), 13, 11, 1.0, center=(0.2, 0.1, -0.3))
        geo = I.ViewGeometry("parallel", np.concatenate([t.src, extra.src]),
                             np.concatenate([t.det_center, extra.det_center]), np.concatenate([t.det_u, extra.det_u]),
                             np.concatenate([t.det_v, extra.det_v]), 13, 11)
    assert geo.n_views > 48
    y = rng.uniform(0, 1, geo.n_rays)
    got = gpu_adjoint(env, dims, origin, geo, y, 3, form=2)
    ref = orc.adjoint(3, dims, origin, y.astype(np.float32).astype(np.float64), oracle_geom(orc, geo))
    assert np.isfinite(got).all()
    assert rel_l2(got, ref) <= TOL, rel_l2(got, ref)


def test_adjoint_coarse_and_close_geometries(env, orc):
    """The scatter adjoint on a coarse detector (pixels much larger than a
    cell: one ray per several bases) and on a cone whose rays within one
    16 x 8 tile have different dominant axes and mirror signs (source close
    to the grid, 45-degree views)."""
    torch, spl = env
    rng = np.random.default_rng(1300)
    dims = (48, 46, 44)
    origin = I.centred_origin(dims)
    coarse = I.parallel_views(np.array([[0.3, 0.5, 0.8], [0.9, -0.1, 0.4]]), 16, 8, 4.3)
    close = I.helical_cone(3, 30.0, 60.0, 19, 17, 3.0, turns=0.375, table_feed=2.0)
    for geo in (coarse, close):
        y = rng.uniform(0, 1, geo.n_rays)
        got = gpu_adjoint(env, dims, origin, geo, y, 3, form=2)
        ref = orc.adjoint(3, dims, origin, y.astype(np.float32).astype(np.float64), oracle_geom(orc, geo))
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, rel_l2(got, ref)


def test_unprepared_basis_is_refused(env):
    """spl_forward / spl_adjoint allocate nothing: through the C ABI, a basis
    whose plane matrices (or footprint tables) the geometry has not built is
    refused with SPL_ERR_STATE until spl_prepare has run; a geometry that
    needs nothing (cone views) runs without it."""
    import ctypes as C

    torch, spl = env
    L = spl.lib()
    origin = I.centred_origin(DIMS)
    st = torch.cuda.current_stream().cuda_stream
    g = spl.Geometry(DIMS, origin, tilt_geometry(2))
    c = torch.ones(g.coeff_shape, dtype=torch.float32, device="cuda")
    y = torch.zeros(g.n_rays, dtype=torch.float32, device="cuda")
    for mode in (spl.SPL_FP_QUAD, spl.SPL_FP_TABLE):
        b = spl.basis(3, mode)
        assert L.spl_forward(g.handle, C.byref(b), spl._ptr(c), spl._ptr(y), C.c_void_p(st)) == 6
        assert L.spl_adjoint(g.handle, C.byref(b), spl._ptr(y), spl._ptr(c), C.c_void_p(st)) == 6
        assert b"spl_prepare" in L.spl_last_error()
        assert L.spl_prepare(g.handle, C.byref(b), C.c_void_p(st)) == 0
        assert L.spl_forward(g.handle, C.byref(b), spl._ptr(c), spl._ptr(y), C.c_void_p(st)) == 0
    torch.cuda.synchronize()
    g.status()
    assert float(y.abs().max()) > 0
    gc = spl.Geometry(DIMS, origin, cone_geometry())
    yc = torch.zeros(gc.n_rays, dtype=torch.float32, device="cuda")
    b = spl.basis(3)
    assert L.spl_forward(gc.handle, C.byref(b), spl._ptr(c), spl._ptr(yc), C.c_void_p(st)) == 0
    torch.cuda.synchronize()
    gc.status()


def test_cuda_graph_capture_of_mixed_geometry(env):
    """A forward and an adjoint of a geometry whose separable views run on the
    geometry's side stream beside the march, captured into a CUDA graph on
    the caller's stream and replayed: the fork and join keep the graph one
    ordered operation, and the replay reproduces the eager results."""
    torch, spl = env
    rng = np.random.default_rng(1777)
    origin = I.centred_origin(DIMS)
    geo = tilt_geometry(2)
    g = spl.Geometry(DIMS, origin, geo)
    bas = spl.basis(3)
    c = torch.tensor(rng.normal(size=DIMS[::-1]).astype(np.float32), device="cuda")
    y_in = torch.tensor(rng.normal(size=geo.n_rays).astype(np.float32), device="cuda")
    y_e = torch.empty(g.n_rays, device="cuda")
    c_e = torch.empty(g.coeff_shape, device="cuda")
    spl.prepare(g, bas)
    spl.forward(g, c, y_e, bas)  # eager: also builds what the geometry needs
    spl.adjoint(g, y_in, c_e, bas)
    torch.cuda.synchronize()
    y_g = torch.full((g.n_rays,), float("nan"), device="cuda")
    c_g = torch.full(g.coeff_shape, float("nan"), device="cuda")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph):
            spl.forward(g, c, y_g, bas)
            spl.adjoint(g, y_in, c_g, bas)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        y_g.fill_(float("nan"))
        c_g.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        g.status()
        assert torch.isfinite(y_g).all() and torch.isfinite(c_g).all()
        assert torch.allclose(y_g, y_e, rtol=0, atol=1e-5 * float(y_e.abs().max()))
        assert torch.allclose(c_g, c_e, rtol=0, atol=1e-5 * float(c_e.abs().max()))
