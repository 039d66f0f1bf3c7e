"""Autograd wrapper and CGLS reconstruction on the GPU operators.

* the backward of SplineXray is the matched adjoint (and vice versa);
* the gradient of 1/2 ||A c - y||^2 matches the oracle gradient
  A^T (A c - y) and a finite difference (the loss is quadratic, so central
  differences are exact up to rounding);
* CGLS iterates match an FP64 CGLS on the oracle operators, and the
  residual norm never increases.
"""
import numpy as np
import pytest

from paper_2511_11078_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (20, 18, 17)


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import recon, spl

    B.build()
    spl.lib()
    return torch, spl, recon


def oracle_geom(orc, geo):
    return orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                        nu=geo.nu, nv=geo.nv)


def setup(env, seed=3000):
    torch, spl, recon = env
    rng = np.random.default_rng(seed)
    geo = I.parallel_views(I.random_directions(rng, 12), 23, 21, 1.0, center=(0.11, -0.07, 0.05))
    origin = I.centred_origin(DIMS)
    g = spl.Geometry(DIMS, origin, geo)
    proj = recon.Projector(g, 3)
    return rng, geo, origin, g, proj


def test_autograd_backward_is_adjoint(env, orc):
    torch, spl, recon = env
    rng, geo, origin, g, proj = setup(env)
    c = torch.tensor(rng.normal(size=DIMS[::-1]).astype(np.float32), device="cuda", requires_grad=True)
    y_obs = torch.tensor(rng.normal(size=g.shape).astype(np.float32), device="cuda")
    y = recon.project(c, proj)
    loss = 0.5 * ((y - y_obs) ** 2).sum()
    loss.backward()
    direct = proj.adjoint((y - y_obs).detach())
    # same kernel; float atomics add in a run-dependent order
    assert torch.allclose(c.grad, direct, rtol=1e-5, atol=1e-5 * float(direct.abs().max()))
    # oracle gradient A^T (A c - y)
    og = oracle_geom(orc, geo)
    c64 = c.detach().cpu().numpy().astype(np.float64)
    res = orc.forward(3, DIMS, origin, c64, og) - y_obs.cpu().numpy().astype(np.float64).reshape(-1)
    gref = orc.adjoint(3, DIMS, origin, res, og)
    got = c.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - gref) <= 1e-5 * np.linalg.norm(gref)
    # transpose operator: backward is the forward projection
    yv = torch.tensor(rng.normal(size=g.shape).astype(np.float32), device="cuda", requires_grad=True)
    cb = recon.backproject(yv, proj)
    w = torch.tensor(rng.normal(size=DIMS[::-1]).astype(np.float32), device="cuda")
    (cb * w).sum().backward()
    assert torch.equal(yv.grad, proj.forward(w))  # the forward is deterministic


def test_loss_gradient_finite_difference(env):
    torch, spl, recon = env
    rng, geo, origin, g, proj = setup(env, 3100)
    c = torch.tensor(rng.uniform(0, 1, size=DIMS[::-1]).astype(np.float32), device="cuda", requires_grad=True)
    y_obs = torch.tensor(rng.uniform(0, 5, size=g.shape).astype(np.float32), device="cuda")

    def loss64(cv):
        y = proj.forward(cv).double()
        return 0.5 * float(((y - y_obs.double()) ** 2).sum())

    y = recon.project(c, proj)
    (0.5 * ((y - y_obs) ** 2).sum()).backward()
    v = torch.tensor(rng.normal(size=DIMS[::-1]).astype(np.float32), device="cuda")
    eps = 0.25
    fd = (loss64(c.detach() + eps * v) - loss64(c.detach() - eps * v)) / (2 * eps)
    an = float((c.grad.double() * v.double()).sum())
    assert abs(fd - an) <= 1e-4 * abs(an), (fd, an)


def test_cgls_matches_fp64_cgls(env, orc):
    torch, spl, recon = env
    import oracle.cgls as OC

    rng, geo, origin, g, proj = setup(env, 3200)
    og = oracle_geom(orc, geo)
    ell = I.random_ellipsoids(rng, DIMS, 4, (2.0, 6.0))
    c_true = I.prefilter(I.rasterize(ell, DIMS), 3).astype(np.float32)
    y = orc.forward(3, DIMS, origin, c_true.astype(np.float64), og)
    y = (y + 0.01 * y.max() * rng.normal(size=y.shape)).astype(np.float32)
    iters = 6
    xs, res = OC.cgls(lambda x: orc.forward(3, DIMS, origin, x, og),
                      lambda r: orc.adjoint(3, DIMS, origin, r, og), y.astype(np.float64), iters)
    cg = recon.CGLS(proj, torch.tensor(y.reshape(g.shape), device="cuda"))
    norms = [cg.residual_norm()]
    for k in range(iters):
        cg.step()
        norms.append(cg.residual_norm())
        xk = cg.x.cpu().numpy().astype(np.float64)
        err = np.linalg.norm(xk - xs[k]) / np.linalg.norm(xs[k])
        assert err <= 1e-4, (k, err)
        assert abs(norms[-1] - res[k]) <= 1e-4 * res[k]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(norms, norms[1:]))
