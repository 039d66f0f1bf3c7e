"""The learned footprint f_theta on the GPU (Sec. 2.2, Algorithm 1).

* evaluation (BF16 tensor-core kernel) against the FP64 oracle MLP under the
  same precision contract (BF16 weights and hidden activations into the
  64x64 layers, FP32 elsewhere);
* gradients of the L2 loss against the oracle gradient of the same
  contract (roundings passed straight through);
* the Algorithm 1 sampler, training progress, and the MLP-footprint
  projector against the oracle's Algorithm 2 with f_theta.

Tolerances.  The contract rounds the hidden activations to BF16, which is
discontinuous: a pre-activation that lies within FP32 rounding of a BF16
rounding boundary may round to the neighbouring BF16 value on the GPU (one
step, 2^-8 to 2^-7 of the activation), and the row then differs by the
effect of that step on f.  Which rows flip depends on the order of the FP32
sums, so the largest difference over many rows measures the flips, not the
arithmetic.  Evaluation: median |diff| <= 1e-5 of max |f| (the arithmetic),
at most 0.5 % of the rows beyond 1e-4 of max |f| (flips are rare: about
0.1 % measured), and every such row explained by a flip: the GPU value lies
within 1e-4 of max |f| of the oracle's output with one hidden activation
that sits within 2^-16 (relative) of a BF16 rounding boundary rounded to its
other neighbour.  2^-16 bounds the GPU's FP32 error in an activation (a
64-term FP32 dot product, the bias, and the SiLU's approximate exponential
and reciprocal, each a few 2^-24 relative) with margin.  Gradients and
projections: relative L2 <= 2e-3.
"""
import numpy as np
import pytest

from paper_2511_11078_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIZES = [5, 64, 64, 64, 1]


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import learn, spl

    B.build()
    spl.lib()
    return torch, spl, learn


def random_params(rng, scale=1.0):
    # fan-in scaled weights, biases of the same order (a generic network)
    parts = []
    for i in range(4):
        fi, fo = SIZES[i], SIZES[i + 1]
        parts.append(rng.normal(size=fo * fi) * scale / np.sqrt(fi))
        parts.append(rng.normal(size=fo) * 0.3)
    return np.concatenate(parts).astype(np.float32)


FLIP_EPS = 2.0 ** -16


def assert_matches_contract(orc, prm, X, got, ref):
    """median within 1e-5 of max |f|; rows beyond 1e-4 rare, each one the
    oracle's output with one near-boundary activation rounded the other way"""
    fmax = np.max(np.abs(ref))
    d = np.abs(got - ref)
    assert np.median(d) <= 1e-5 * fmax
    far = np.nonzero(d > 1e-4 * fmax)[0]
    assert far.size <= max(1, 0.005 * d.size), far.size
    for r in far:
        alts = orc.mlp_flip_variants(SIZES, prm.astype(np.float64), X[r].astype(np.float64), FLIP_EPS)
        assert alts.size > 0, ("row differs without a near-boundary activation", r, d[r] / fmax)
        assert np.min(np.abs(alts - got[r])) <= 1e-4 * fmax, ("no single flip explains row", r, d[r] / fmax)


def random_features(rng, n):
    w = np.sort(np.abs(I.random_directions(rng, n)), axis=1)
    uv = rng.uniform(-1, 1, (n, 2))
    return np.concatenate([w, uv], axis=1).astype(np.float32)


def test_mlp_eval_matches_oracle(env, orc):
    torch, spl, learn = env
    rng = np.random.default_rng(5000)
    m = spl.Mlp(3, max_batch=1024, seed=1)
    prm = random_params(rng)
    m.set_params(prm)
    X = random_features(rng, 10007)  # ragged tail: not a multiple of 16
    out = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    m.eval(torch.tensor(X, device="cuda"), out)
    ref = orc.mlp_forward(SIZES, prm.astype(np.float64), X.astype(np.float64), mode=1)
    got = out.cpu().numpy().astype(np.float64)
    assert_matches_contract(orc, prm, X, got, ref)
    m.status()
    # against the FP64 network the BF16 contract is a small, nonzero change
    ref0 = orc.mlp_forward(SIZES, prm.astype(np.float64), X.astype(np.float64), mode=0)
    assert 0 < np.max(np.abs(got - ref0)) <= 5e-2 * np.max(np.abs(ref0))


@pytest.mark.parametrize("count", [1, 127, 129, 200003])
def test_mlp_eval_tile_tails_and_many_tiles(env, orc, count):
    # The evaluation runs 128-row tiles on a grid of at most 608 CTAs: one
    # row, a tile minus one, a tile plus one, and enough rows for every CTA
    # to run several tiles (the tensor-core completion barrier then cycles
    # through its phases).
    torch, spl, learn = env
    rng = np.random.default_rng(5100 + count)
    m = spl.Mlp(3, max_batch=1024, seed=2)
    prm = random_params(rng)
    m.set_params(prm)
    X = random_features(rng, count)
    out = torch.full((count,), float("nan"), dtype=torch.float32, device="cuda")
    m.eval(torch.tensor(X, device="cuda"), out)
    ref = orc.mlp_forward(SIZES, prm.astype(np.float64), X.astype(np.float64), mode=1)
    got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    assert_matches_contract(orc, prm, X, got, ref)
    m.status()


def test_mlp_params_roundtrip_and_init(env):
    torch, spl, learn = env
    m = spl.Mlp(2, max_batch=64, seed=123)
    p0 = m.get_params()
    assert p0.shape == (spl.MLP_PARAMS,) and np.all(np.isfinite(p0))
    # seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation
    assert np.max(np.abs(p0[:320])) <= 1 / np.sqrt(5) + 1e-7 and np.max(np.abs(p0[384:4480])) <= 0.125 + 1e-7
    assert np.array_equal(p0, spl.Mlp(2, max_batch=64, seed=123).get_params())
    rng = np.random.default_rng(1)
    p1 = rng.normal(size=spl.MLP_PARAMS).astype(np.float32)
    m.set_params(p1)
    assert np.array_equal(m.get_params(), p1)
    with pytest.raises(spl.SplError):
        bad = p1.copy()
        bad[7] = np.nan
        m.set_params(bad)


def test_mlp_checkpoint_resumes_training_exactly(env, tmp_path):
    """spl_mlp_save / spl_mlp_load carry the parameters, the Adam moments
    and the step count: a network restored from a checkpoint and trained on
    the same batches ends bit-identical to the one that kept training; a
    checkpoint of another degree is refused."""
    torch, spl, learn = env
    data = learn.FootprintSet(3, 1 << 14, seed=61)
    a = spl.Mlp(3, max_batch=1024, seed=8)
    batches = [(data.feat[i * 1024:(i + 1) * 1024], data.label[i * 1024:(i + 1) * 1024]) for i in range(12)]
    for f, t in batches[:6]:
        a.train_step(f, t, 2e-3)
    path = str(tmp_path / "f_theta.ckpt")
    a.save(path)
    for f, t in batches[6:]:
        a.train_step(f, t, 2e-3)
    b = spl.Mlp(3, max_batch=1024, seed=99)
    b.load(path)
    for f, t in batches[6:]:
        b.train_step(f, t, 2e-3)
    torch.cuda.synchronize()
    pa, pb = a.get_params(), b.get_params()
    assert np.array_equal(pa, pb)
    # without the Adam state (parameters only) the continuation differs
    c = spl.Mlp(3, max_batch=1024, seed=99)
    c.load(path)
    c.set_params(c.get_params())  # resets Adam
    for f, t in batches[6:]:
        c.train_step(f, t, 2e-3)
    assert not np.array_equal(c.get_params(), pa)
    a.status()
    b.status()
    with pytest.raises(spl.SplError):
        spl.Mlp(2, max_batch=64, seed=1).load(path)
    with open(path, "r+b") as fh:  # a truncated file is refused
        fh.truncate(100)
    with pytest.raises(spl.SplError):
        b.load(path)


@pytest.mark.parametrize("batch", [16, 1000, 4099])
def test_mlp_gradient_matches_oracle(env, orc, batch):
    torch, spl, learn = env
    rng = np.random.default_rng(5100 + batch)
    m = spl.Mlp(3, max_batch=4096 + 16, seed=2)
    prm = random_params(rng, 0.8)
    m.set_params(prm)
    X = random_features(rng, batch)
    Y = rng.normal(size=batch).astype(np.float32) * 0.2
    grad = torch.empty(spl.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    m.grad(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), grad, loss)
    L, gref = orc.mlp_loss_grad(SIZES, prm.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), mode=1)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - L) <= 1e-3 * L
    assert np.linalg.norm(g - gref) <= 2e-3 * np.linalg.norm(gref)
    # every layer's gradient individually
    offs = [0, 384, 4544, 8704, 8769]
    for a, b in zip(offs[:-1], offs[1:]):
        assert np.linalg.norm(g[a:b] - gref[a:b]) <= 5e-3 * np.linalg.norm(gref[a:b]) + 1e-9


@pytest.mark.parametrize("batch", [100, 8192])
def test_mlp_gradient_parameter_groups(env, orc, batch):
    # Each weight matrix and each bias vector on its own, so that an error in
    # a small group (a bias, the output layer) cannot hide in a layer's norm;
    # batch 8192 spans many weight-gradient chunks and reduction blocks.
    torch, spl, learn = env
    rng = np.random.default_rng(5300 + batch)
    m = spl.Mlp(3, max_batch=8192, seed=3)
    prm = random_params(rng, 0.8)
    m.set_params(prm)
    X = random_features(rng, batch)
    Y = rng.normal(size=batch).astype(np.float32) * 0.2
    grad = torch.empty(spl.MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    m.grad(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), grad, loss)
    L, gref = orc.mlp_loss_grad(SIZES, prm.astype(np.float64), X.astype(np.float64), Y.astype(np.float64), mode=1)
    g = grad.cpu().numpy().astype(np.float64)
    groups = [(0, 320), (320, 384), (384, 4480), (4480, 4544), (4544, 8640), (8640, 8704), (8704, 8768), (8768, 8769)]
    for a, b in groups:
        assert np.linalg.norm(g[a:b] - gref[a:b]) <= 1e-4 * np.linalg.norm(gref[a:b]) + 1e-12, (a, b)


def test_sampler_distribution(env, orc):
    torch, spl, learn = env
    n = 200000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    normals = torch.randn((n, 3), generator=gen, device="cuda")
    uniforms = torch.rand((n, 2), generator=gen, device="cuda")
    w = torch.empty((n, 3), device="cuda")
    p = torch.empty((n, 3), device="cuda")
    spl.footprint_samples(3, normals, uniforms, w, p)
    w, p = w.cpu().numpy().astype(np.float64), p.cpu().numpy().astype(np.float64)
    nz = normals.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(w, nz / np.linalg.norm(nz, axis=1, keepdims=True), atol=1e-6)
    assert np.max(np.abs(np.sum(w * p, axis=1))) < 1e-5          # p in H_w
    r = np.linalg.norm(p, axis=1)
    R = np.sqrt(3.0) * 2.0
    assert r.max() <= R * (1 + 1e-6)
    # uniform in the disc: P(r < R/2) = 1/4
    assert abs(np.mean(r < R / 2) - 0.25) < 0.005
    # uniform on the sphere: mean of w ~ 0, mean of w_z^2 = 1/3
    assert np.all(np.abs(w.mean(0)) < 0.01) and abs(np.mean(w[:, 2] ** 2) - 1 / 3) < 0.005


def test_training_reduces_error(env):
    """A few hundred Adam steps on exact-footprint samples reduce the error
    against the exact footprint well below the untrained network's."""
    torch, spl, learn = env
    data = learn.FootprintSet(3, 1 << 16, seed=11)
    val = learn.FootprintSet(3, 1 << 13, seed=12)
    m = spl.Mlp(3, max_batch=4096, seed=3)
    e0 = learn.evaluate(m, val)
    hist = learn.train(m, data, steps=400, batch=4096, lr0=3e-3, lr_min=1e-4, val=val, log_every=100)
    e1 = learn.evaluate(m, val)
    assert hist[-1]["loss"] < 0.05 * hist[0]["loss"]
    assert e1["rms"] < 0.1 * e0["rms"]
    assert e1["max_abs"] < 0.2 * e0["max_abs"]


def _trained(env, degree=3):
    torch, spl, learn = env
    data = learn.FootprintSet(degree, 1 << 16, seed=21)
    m = spl.Mlp(degree, max_batch=4096, seed=4)
    learn.train(m, data, steps=1500, batch=4096, lr0=3e-3, lr_min=1e-5)
    return m


DIMS = (12, 11, 10)


def test_mlp_projector_matches_oracle(env, orc):
    torch, spl, learn = env
    m = _trained(env)
    rng = np.random.default_rng(5300)
    origin = I.centred_origin(DIMS)
    geo = I.parallel_views(I.random_directions(rng, 3), 13, 12, 1.0, center=(0.1, -0.2, 0.05))
    g = spl.Geometry(DIMS, origin, geo)
    c = rng.uniform(0, 1, size=DIMS[::-1]).astype(np.float32)
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    spl.forward(g, torch.tensor(c, device="cuda"), y, spl.basis(3, spl.SPL_FP_MLP, m))
    g.status()
    og = orc.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                      nu=geo.nu, nv=geo.nv)
    prm = m.get_params().astype(np.float64)
    yref = orc.forward_mlp(3, DIMS, origin, c.astype(np.float64), og, SIZES, prm, mode=1)
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - yref) <= 2e-3 * np.linalg.norm(yref)
    # the exact operator differs from the learned one by the MLP's error
    yq = orc.forward(3, DIMS, origin, c.astype(np.float64), og)
    assert np.linalg.norm(got - yq) <= 0.05 * np.linalg.norm(yq)


def test_mlp_projector_full_size_sampled(env, orc):
    """The learned-footprint projector on the benchmark's 128^3 cubic tilt
    workload (all 244 views, the launch the benchmark times): sampled rays
    against the oracle's BF16-contract projector, each sampled ray evaluated
    as a one-pixel view with the same direction and pixel centre."""
    torch, spl, learn = env
    m = _trained(env)
    wl = I.workload_tilt(3)
    g = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    y = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
    spl.forward(g, torch.tensor(wl.coeffs, device="cuda"), y, spl.basis(3, spl.SPL_FP_MLP, m))
    g.status()
    rng = np.random.default_rng(5350)
    rays = np.sort(rng.choice(g.n_rays, 24, replace=False))
    got = y.cpu().numpy()[rays].astype(np.float64)
    prm = m.get_params().astype(np.float64)
    geo = wl.geometry
    per = geo.nu * geo.nv
    ref = np.zeros(len(rays))
    for t, r in enumerate(rays):
        k = int(r // per)
        iv, iu = divmod(int(r - k * per), geo.nu)
        a, b = iu - 0.5 * (geo.nu - 1), iv - 0.5 * (geo.nv - 1)
        q = geo.det_center[k] + a * geo.det_u[k] + b * geo.det_v[k]
        og = orc.Geometry("parallel", direction=geo.src[k:k + 1], det_center=q[None], det_u=geo.det_u[k:k + 1],
                          det_v=geo.det_v[k:k + 1], nu=1, nv=1)
        ref[t] = orc.forward_mlp(3, wl.dims, wl.origin, wl.coeffs.astype(np.float64), og, SIZES, prm, mode=1)[0]
    assert np.linalg.norm(got - ref) <= 2e-3 * np.linalg.norm(ref), np.linalg.norm(got - ref) / np.linalg.norm(ref)


def test_mlp_projector_adjointness(env):
    torch, spl, learn = env
    m = _trained(env)
    rng = np.random.default_rng(5400)
    origin = I.centred_origin(DIMS)
    for geo in (I.parallel_views(I.random_directions(rng, 4), 15, 14, 1.0),
                I.helical_cone(3, 40.0, 60.0, 17, 15, 1.3, turns=0.7, table_feed=3.0)):
        g = spl.Geometry(DIMS, origin, geo)
        b = spl.basis(3, spl.SPL_FP_MLP, m)
        c = torch.tensor(rng.normal(size=DIMS[::-1]).astype(np.float32), device="cuda")
        yv = torch.tensor(rng.normal(size=g.n_rays).astype(np.float32), device="cuda")
        Ac = torch.empty(g.n_rays, dtype=torch.float32, device="cuda")
        ATy = torch.empty(g.coeff_shape, dtype=torch.float32, device="cuda")
        spl.forward(g, c, Ac, b)
        spl.adjoint(g, yv, ATy, b)
        g.status()
        lhs = float((Ac.double() * yv.double()).sum())
        rhs = float((c.double() * ATy.double()).sum())
        assert abs(lhs - rhs) <= 1e-5 * float(Ac.double().norm() * yv.double().norm())


def test_mlp_footprint_support_mask(env):
    """f_theta is kept only on the exact support: zero where the line misses
    the basis."""
    torch, spl, learn = env
    m = spl.Mlp(3, max_batch=64, seed=9)
    w = torch.tensor([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [1.0, 1.0, 1.0]], device="cuda") / torch.tensor(
        [[1.0], [1.0], [3 ** 0.5]], device="cuda")
    p = torch.tensor([[2.5, 0.0, 0.0], [1.0, 1.0, 0.0], [3.0, -3.0, 0.0]], device="cuda")
    out = torch.empty(3, device="cuda")
    spl.footprint(spl.basis(3, spl.SPL_FP_MLP, m), w, p, out)
    o = out.cpu().numpy()
    assert o[0] == 0.0 and o[2] == 0.0 and o[1] != 0.0


def test_trained_network_gain(env, orc):
    """What training f_theta gains: its footprint error against the exact
    footprint falls far below the untrained network's, and the projector
    built on it reproduces the exact operator's projections to well under a
    percent.  What it costs on this GPU: footprint evaluations per second of
    the tensor-core MLP next to the exact per-pair quadrature (printed; the
    exact evaluator is the faster one here, see the measurement notes)."""
    import time

    torch, spl, learn = env
    data = learn.FootprintSet(3, 1 << 20, seed=41)
    val = learn.FootprintSet(3, 1 << 16, seed=42)
    m = spl.Mlp(3, max_batch=8192, seed=6)
    before = learn.evaluate(m, val)
    learn.train(m, data, steps=3000, batch=8192, lr0=3e-3, lr_min=1e-6)
    after = learn.evaluate(m, val)
    assert after["rms"] < 0.02 * before["rms"]
    assert after["max_abs_rel_peak"] < 0.05
    # projections of a smooth volume: learned vs exact operator
    rng = np.random.default_rng(43)
    dims = (24, 22, 20)
    origin = I.centred_origin(dims)
    geo = I.parallel_views(I.random_directions(rng, 6), 31, 29, 1.0)
    g = spl.Geometry(dims, origin, geo)
    ell = I.random_ellipsoids(rng, dims, 5, (3.0, 7.0))
    c = torch.tensor(I.prefilter(I.rasterize(ell, dims), 3).astype(np.float32), device="cuda")
    yq = torch.empty(g.n_rays, device="cuda")
    ym = torch.empty(g.n_rays, device="cuda")
    spl.forward(g, c, yq, spl.basis(3))
    spl.forward(g, c, ym, spl.basis(3, spl.SPL_FP_MLP, m))
    g.status()
    assert float((ym - yq).norm() / yq.norm()) < 1e-2
    # footprint evaluations per second, same samples
    rates = {}
    for name, b in (("exact", spl.basis(3)), ("mlp", spl.basis(3, spl.SPL_FP_MLP, m))):
        out = torch.empty(data.count, device="cuda")
        spl.footprint(b, data.omega, data.p, out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            spl.footprint(b, data.omega, data.p, out)
        torch.cuda.synchronize()
        rates[name] = 5 * data.count / (time.perf_counter() - t0)
    print("trained f_theta: max|err|/peak %.2e (untrained %.2e), rms %.2e; footprints/s exact %.3g, mlp %.3g"
          % (after["max_abs_rel_peak"], before["max_abs_rel_peak"], after["rms"], rates["exact"], rates["mlp"]))
