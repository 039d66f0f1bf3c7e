"""Spline vs voxel reconstruction (the experiment of Sec. 3 / Fig. 4).

The paper reconstructs a BrainWeb head volume (180 x 180 x 50) from 200
cone-beam views on a 180 x 50 detector, with Gaussian
noise of variance 1e-3, by 50 conjugate-gradient iterations of
non-regularised least squares, once with quadratic B-splines and once with
voxels (the classic DDA), and reports the PSNR of both.  BrainWeb is not
available here: a head-like ellipsoid phantom of the same size stands in
for it, and its data are the exact line integrals of the continuous
ellipsoids (not projections of either discrete model), so neither basis is
favoured by the data.  PSNR compares the reconstructed function sampled at
the grid points with the phantom sampled there:
PSNR = 10 log10(max(ref)^2 / MSE).

Run: python -m paper_2511_11078_gb300.experiment [--iters 50] [--degree 2]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import inputs as I
from . import spl
from .recon import CGLS, Projector

# beta^n at the integers 0 and +-1 (sampling a spline at the grid points)
_TAPS = {0: (1.0, 0.0), 1: (1.0, 0.0), 2: (0.75, 0.125), 3: (2.0 / 3.0, 1.0 / 6.0)}


def head_phantom(rng, dims):
    """A head-like phantom: an outer ellipsoidal skull shell, brain tissue
    and a few inner structures (densities in [0, 1])."""
    nx, ny, nz = dims
    ext = np.array([nx, ny, nz], dtype=np.float64) - 1.0
    centers, axes, rots, dens = [], [], [], []

    def add(c, a, R, d):
        centers.append(c)
        axes.append(a)
        rots.append(R)
        dens.append(d)

    eye = np.eye(3)
    add(np.zeros(3), 0.46 * ext, eye, 0.8)        # skull (outer)
    add(np.zeros(3), 0.42 * ext, eye, -0.6)       # skull (inner cut)
    Rr = I.random_rotations(rng, 10)
    for k in range(10):
        c = rng.uniform(-0.25, 0.25, 3) * ext
        a = rng.uniform(0.03, 0.12, 3) * ext[:3]
        a[2] = min(a[2], 0.3 * ext[2])
        add(c, a, Rr[k], rng.uniform(0.1, 0.5))
    return I.Ellipsoids(np.array(centers), np.array(axes), np.array(rots), np.array(dens))


def view_rays(geo):
    """World rays (s, w) of a view geometry, ray order of the projections."""
    V, nu, nv = geo.n_views, geo.nu, geo.nv
    a = (np.arange(nu) - 0.5 * (nu - 1))[None, None, :, None]
    b = (np.arange(nv) - 0.5 * (nv - 1))[None, :, None, None]
    q = (geo.det_center[:, None, None, :] + a * geo.det_u[:, None, None, :] + b * geo.det_v[:, None, None, :])
    if geo.kind == "parallel":
        w = np.broadcast_to(geo.src[:, None, None, :], q.shape)
        s = q
    else:
        s = np.broadcast_to(geo.src[:, None, None, :], q.shape)
        w = q - s
    w = w / np.linalg.norm(w, axis=-1, keepdims=True)
    return np.ascontiguousarray(s.reshape(-1, 3)), np.ascontiguousarray(w.reshape(-1, 3))


def sample_spline(c, degree):
    """f at the grid points: c filtered by beta^n at the integers per axis."""
    t0, t1 = _TAPS[degree]
    f = np.array(c, dtype=np.float64)
    if t1 == 0.0:
        return f
    for ax in range(3):
        g = t0 * f
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        g[tuple(sl_hi)] += t1 * f[tuple(sl_lo)]
        g[tuple(sl_lo)] += t1 * f[tuple(sl_hi)]
        f = g
    return f


def psnr(f, ref):
    mse = float(np.mean((f - ref) ** 2))
    return 10.0 * math.log10(float(ref.max()) ** 2 / mse)


def run(dims=(180, 180, 50), n_views=200, det=(180, 50), iters=50, degrees=(2, 0), noise_var=1e-3, seed=7,
        sod_factor=4.0, device="cuda"):
    rng = np.random.default_rng(I.SEED_BASE + 100 + seed)
    ell = head_phantom(rng, dims)
    ref = I.rasterize(ell, dims)
    # cone beam, 200 views on a circle about the axis of the 50 slices (the
    # only rotation axis for which a 180 x 50 detector holds the whole
    # 180 x 180 x 50 volume); flat detector at twice the source distance,
    # pitch chosen so the volume's projection fits
    L = float(max(dims))
    sod, sdd = sod_factor * L, 2.0 * sod_factor * L
    pitch = 1.1 * (sdd / sod) * max(dims[0] / det[0], dims[2] / det[1])
    geo = I.circular_cone(n_views, sod, sdd, det[0], det[1], pitch)
    s, w = view_rays(geo)
    y = I.ellipsoid_line_integrals(ell, s, w)
    y = y + math.sqrt(noise_var) * rng.standard_normal(y.shape)
    g = spl.Geometry(dims, I.centred_origin(dims), geo)
    yt = torch.tensor(y.astype(np.float32).reshape(g.shape), device=device)
    out = {"dims": list(dims), "views": n_views, "detector": list(det), "iters": iters, "noise_var": noise_var}
    for n in degrees:
        proj = Projector(g, n)
        cg = CGLS(proj, yt)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        cg.run(iters)
        t1.record()
        torch.cuda.synchronize()
        g.status()
        c = cg.x.cpu().numpy()
        f = sample_spline(c, n)
        out["degree_%d" % n] = {"psnr_db": psnr(f, ref), "residual": cg.residual_norm(),
                                "s_per_iter": t0.elapsed_time(t1) / 1e3 / iters}
    if len(degrees) == 2:
        out["psnr_gap_db"] = out["degree_%d" % degrees[0]]["psnr_db"] - out["degree_%d" % degrees[1]]["psnr_db"]
    return out


def cylinder_mask(dims):
    """Grid points inside the cylinder inscribed in the grid about e3 (the
    cone-beam detectors of the workloads truncate the volume's corners)."""
    nx, ny, nz = dims
    org = I.centred_origin(dims)
    x = org[0] + np.arange(nx)
    y = org[1] + np.arange(ny)
    r = 0.5 * (min(nx, ny) - 1)
    inside = (x[None, :] ** 2 + y[:, None] ** 2) <= r * r
    return np.broadcast_to(inside[None, :, :], (nz, ny, nx))


def mlp_vs_quadrature(mlp, iters=10, views=None, noise=0.01, device="cuda"):
    """The learned footprint inside least squares (Sec. 2.2 used in Eq. 5)
    beside the exact quadrature, on the 256^3 circular cone-beam workload:
    data y = A c_true + Gaussian noise (sigma = `noise` times max A c_true),
    `iters` CGLS iterations with each footprint form, PSNR of the
    reconstructed spline sampled at the grid points against the phantom's
    spline c_true sampled there, inside the inscribed cylinder.  Returns the
    PSNRs, their difference (the loss from the learned footprint) and the
    seconds per iteration of each form."""
    wl = I.workload_cone()
    geo = wl.geometry if views is None else wl.geometry.subset_views(views)
    g = spl.Geometry(wl.dims, wl.origin, geo)
    c_true = torch.tensor(wl.coeffs, device=device)
    pq = Projector(g, 3)
    y = pq.forward(c_true)
    gen = torch.Generator(device=device)
    gen.manual_seed(I.SEED_BASE + 40)
    y = y + noise * float(y.max()) * torch.randn(y.shape, generator=gen, device=device)
    ref = sample_spline(wl.coeffs.astype(np.float64), 3)
    mask = cylinder_mask(wl.dims)
    out = {"workload": wl.name + "-cubic", "views": geo.n_views, "iters": iters, "noise_sigma_rel_max": noise}
    for name, proj in (("quad", pq), ("mlp", Projector(g, 3, spl.SPL_FP_MLP, mlp))):
        cg = CGLS(proj, y)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        cg.run(iters)
        t1.record()
        torch.cuda.synchronize()
        g.status()
        f = sample_spline(cg.x.cpu().numpy().astype(np.float64), 3)
        out[name] = {"psnr_db": psnr(f[mask], ref[mask]), "residual": cg.residual_norm(),
                     "s_per_iter": t0.elapsed_time(t1) / 1e3 / iters}
    out["psnr_loss_db"] = out["quad"]["psnr_db"] - out["mlp"]["psnr_db"]
    return out


def helical_recon(iters=20, checkpoints=(10, 20), noise=0.01, device="cuda"):
    """The least-squares reconstruction of the 512^3 helical cone-beam
    workload (720 views, 768^2 detector) with the exact footprint: data
    y = A c_true + Gaussian noise (sigma = `noise` times max A c_true),
    `iters` CGLS iterations (Eq. 5 on the normal equations, c0 = 0), the
    PSNR of the reconstructed spline sampled at the grid points against the
    phantom's spline sampled there, inside the inscribed cylinder, after the
    iterations listed in `checkpoints`, and the seconds per iteration
    (CUDA events around the iterations only)."""
    wl = I.workload_helical()
    g = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    c_true = torch.tensor(wl.coeffs, device=device)
    proj = Projector(g, 3)
    y = proj.forward(c_true)
    gen = torch.Generator(device=device)
    gen.manual_seed(I.SEED_BASE + 41)
    y = y + noise * float(y.max()) * torch.randn(y.shape, generator=gen, device=device)
    del c_true
    ref = sample_spline(wl.coeffs.astype(np.float64), 3)
    mask = cylinder_mask(wl.dims)
    ref_in = ref[mask]
    del ref
    cg = CGLS(proj, y)
    out = {"workload": wl.name + "-cubic", "views": wl.geometry.n_views, "iters": iters,
           "noise_sigma_rel_max": noise, "psnr_db": {}}
    gpu_ms = 0.0
    for k in range(1, iters + 1):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        cg.step()
        t1.record()
        torch.cuda.synchronize()
        gpu_ms += t0.elapsed_time(t1)
        if k in checkpoints:
            g.status()
            f = sample_spline(cg.x.cpu().numpy().astype(np.float64), 3)
            out["psnr_db"][k] = psnr(f[mask], ref_in)
            del f
    out["residual"] = cg.residual_norm()
    out["s_per_iter"] = gpu_ms / 1e3 / iters
    out["s_total"] = gpu_ms / 1e3
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--degree", type=int, default=2)
    ap.add_argument("--seeds", type=int, default=1)
    ap.add_argument("--mlp-checkpoint", default=None,
                    help="instead: the learned footprint of this checkpoint (spl_mlp_save) against quadrature "
                         "inside CGLS on the 256^3 cone-beam workload, --iters iterations each")
    ap.add_argument("--helical", action="store_true",
                    help="instead: --iters CGLS iterations on the 512^3 helical cone-beam workload (exact footprint)")
    args = ap.parse_args()
    from . import build as B

    B.build()
    if args.helical:
        print(json.dumps(helical_recon(iters=args.iters, checkpoints=(args.iters // 2, args.iters))), flush=True)
        return
    if args.mlp_checkpoint:
        mlp = spl.Mlp(3, max_batch=8192)
        mlp.load(args.mlp_checkpoint)
        print(json.dumps(mlp_vs_quadrature(mlp, iters=args.iters)), flush=True)
        return
    for k in range(args.seeds):
        print(json.dumps(run(iters=args.iters, degrees=(args.degree, 0), seed=k)), flush=True)


if __name__ == "__main__":
    main()
