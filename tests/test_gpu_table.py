"""GPU parity of the footprint-table (splat-form) projector, SPL_FP_TABLE,
through the C ABI, against the oracle's definition of the same approximate
operator (exact footprints at the table nodes, bilinear interpolation, the
exact pair set): relative L2 <= 1e-5, the FP32 bound of the exact path.
Also its distance to the exact operator (second order in the table step)
and its refusal of geometries that have no per-view footprint."""
import numpy as np
import pytest

from paper_2511_11078_gb300 import inputs as I
from test_gpu_parity import DIMS, cone_geometry, oracle_geom, parallel_geometry, rel_l2, tilt_geometry

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import spl

    B.build()
    spl.lib()
    return torch, spl


@pytest.mark.parametrize("geo_kind", ["parallel", "tilt"])
@pytest.mark.parametrize("degree", [1, 2, 3])
def test_table_forward_and_adjoint(env, orc, geo_kind, degree):
    torch, spl = env
    rng = np.random.default_rng(4200 + degree)
    origin = I.centred_origin(DIMS)
    geo = parallel_geometry(rng) if geo_kind == "parallel" else tilt_geometry(2)
    g = spl.Geometry(DIMS, origin, geo)
    c = rng.normal(size=DIMS[::-1]).astype(np.float32)
    y = rng.normal(size=geo.n_rays).astype(np.float32)
    bas = spl.basis(degree, spl.SPL_FP_TABLE)
    yo = torch.full((g.n_rays,), float("nan"), dtype=torch.float32, device="cuda")
    co = torch.full(g.coeff_shape, float("nan"), dtype=torch.float32, device="cuda")
    spl.forward(g, torch.tensor(c, device="cuda"), yo, bas)
    spl.adjoint(g, torch.tensor(y, device="cuda"), co, bas)
    g.status()
    og = oracle_geom(orc, geo)
    yref = orc.forward_table(degree, DIMS, origin, c.astype(np.float64), og)
    cref = orc.adjoint_table(degree, DIMS, origin, y.astype(np.float64), og)
    yg = yo.cpu().numpy().astype(np.float64)
    cg = co.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(yg)) and np.all(np.isfinite(cg))
    assert rel_l2(yg, yref) <= TOL, rel_l2(yg, yref)
    assert rel_l2(cg, cref) <= TOL, rel_l2(cg, cref)
    # the same table values in both directions: <A_T c, y> = <c, A_T^T y>
    lhs, rhs = float(yg @ y.astype(np.float64)), float(np.sum(c.astype(np.float64) * cg))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(yg) * np.linalg.norm(y), (lhs, rhs)
    # and close to the exact operator (h = 1/32: second order)
    yex = orc.forward(degree, DIMS, origin, c.astype(np.float64), og)
    assert rel_l2(yg, yex) <= 2e-3, rel_l2(yg, yex)


def test_table_full_size_sampled(env, orc):
    """128^3 cubic, all 244 views of the tilt-series workload through the
    tables: sampled rays against the oracle's table operator, each sampled
    ray evaluated as a one-pixel view with the same direction, det_u and
    pixel centre (the operator depends on a view only through those)."""
    torch, spl = env
    wl = I.workload_tilt(3)
    g = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    spl.forward(g, torch.tensor(wl.coeffs, device="cuda"), y, spl.basis(3, spl.SPL_FP_TABLE))
    g.status()
    rng = np.random.default_rng(4250)
    rays = np.sort(rng.choice(g.n_rays, 40, replace=False))
    got = y.cpu().numpy()[rays].astype(np.float64)
    ref = np.zeros(len(rays))
    geo = wl.geometry
    per = geo.nu * geo.nv
    for t, r in enumerate(rays):
        k = int(r // per)
        iv, iu = divmod(int(r - k * per), geo.nu)
        a, b = iu - 0.5 * (geo.nu - 1), iv - 0.5 * (geo.nv - 1)
        q = geo.det_center[k] + a * geo.det_u[k] + b * geo.det_v[k]
        one = I.ViewGeometry("parallel", geo.src[k:k + 1], q[None], geo.det_u[k:k + 1], geo.det_v[k:k + 1], 1, 1)
        ref[t] = orc.forward_table(3, wl.dims, wl.origin, wl.coeffs.astype(np.float64), oracle_geom(orc, one))[0]
    assert rel_l2(got, ref) <= TOL, rel_l2(got, ref)


def test_table_refuses_cone_geometry(env):
    torch, spl = env
    g = spl.Geometry(DIMS, I.centred_origin(DIMS), cone_geometry())
    c = torch.zeros(g.coeff_shape, dtype=torch.float32, device="cuda")
    y = torch.zeros(g.n_rays, dtype=torch.float32, device="cuda")
    with pytest.raises(spl.SplError) as ei:
        spl.forward(g, c, y, spl.basis(3, spl.SPL_FP_TABLE))
    assert ei.value.status == 7
