"""Training of the learned footprint f_theta (Algorithm 1, Sec. 2.2).

Samples: directions uniform on the sphere, offsets uniform in the disc of
radius sqrt(3) W of H_w (spl_footprint_samples, random numbers drawn by a
seeded torch generator); labels: the exact footprint (spl_footprint with
the quadrature evaluator, replacing the paper's fine-grid projector);
features: spl_features (canonical direction and frame).  Training: L2 loss,
Adam (spl_mlp_train_step) with cosine learning-rate decay, a held-out set
to measure max-abs and RMS error against the exact footprint.
"""
from __future__ import annotations

import math

import torch

from . import spl

class FootprintSet:
    """`count` exact-footprint samples of Algorithm 1 resident on the GPU.

    The plain set (the defaults) is Algorithm 1's distribution: directions
    uniform on the sphere, offsets uniform in the disc of radius sqrt(3) W.
    Training sets may reshape it (the draws stay the caller's random
    numbers fed to spl_footprint_samples):

    * support_only: keep only samples inside the exact support (nonzero
      label).  The projector multiplies f_theta by the exact support
      indicator, so the values outside are never used; without them the
      loss measures only what the projector sees.
    * axis_fraction: that fraction of the directions is drawn near the six
      coordinate axes (a standard normal plus axis_scale times a random
      signed unit axis, normalised), where the canonical direction sits in
      the chamber's corner w = e3 and the footprint's peak is sharpest.
    * center_power: offsets at radius sqrt(3) W u^(center_power / 2)
      instead of u^(1/2) (u uniform): > 1 draws more samples near the
      footprint's peak at p = 0.
    """

    def __init__(self, degree: int, count: int, seed: int, device="cuda", support_only: bool = False,
                 axis_fraction: float = 0.0, axis_scale: float = 8.0, center_power: float = 1.0):
        self.degree = int(degree)
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        normals = torch.randn((count, 3), generator=gen, device=device)
        uniforms = torch.rand((count, 2), generator=gen, device=device)
        if axis_fraction > 0.0:
            m = int(round(axis_fraction * count))
            axis = torch.randint(0, 3, (m,), generator=gen, device=device)
            sign = torch.randint(0, 2, (m,), generator=gen, device=device).float() * 2.0 - 1.0
            normals[:m].scatter_add_(1, axis[:, None], (axis_scale * sign)[:, None])
        if center_power != 1.0:
            uniforms[:, 0] = uniforms[:, 0].pow(center_power)
        self.omega = torch.empty((count, 3), dtype=torch.float32, device=device)
        self.p = torch.empty((count, 3), dtype=torch.float32, device=device)
        spl.footprint_samples(degree, normals, uniforms, self.omega, self.p)
        self.label = torch.empty(count, dtype=torch.float32, device=device)
        spl.footprint(spl.basis(degree), self.omega, self.p, self.label)
        if support_only:
            keep = torch.nonzero(self.label > 0.0).flatten()
            self.omega = self.omega.index_select(0, keep).contiguous()
            self.p = self.p.index_select(0, keep).contiguous()
            self.label = self.label.index_select(0, keep).contiguous()
        self.count = int(self.label.numel())
        self.feat = torch.empty((self.count, 5), dtype=torch.float32, device=device)
        spl.features(degree, self.omega, self.p, self.feat)

    @property
    def peak(self) -> float:
        return float(self.label.max())


def evaluate(mlp: "spl.Mlp", data: FootprintSet) -> dict:
    """Errors of f_theta (as evaluated by the tensor-core kernel, masked by
    the exact support) against the exact footprint of the samples."""
    out = torch.empty_like(data.label)
    spl.footprint(spl.basis(data.degree, spl.SPL_FP_MLP, mlp), data.omega, data.p, out)
    err = (out - data.label).double()
    peak = data.peak
    return {"max_abs": float(err.abs().max()), "rms": float(err.pow(2).mean().sqrt()), "peak": peak,
            "max_abs_rel_peak": float(err.abs().max()) / peak}


def train(mlp: "spl.Mlp", data: FootprintSet, steps: int, batch: int = 8192, lr0: float = 2e-3,
          lr_min: float = 1e-5, seed: int = 0, val: FootprintSet | None = None, log_every: int = 0,
          callback=None) -> list:
    """Adam on the L2 loss with cosine decay from lr0 to lr_min; minibatches
    are contiguous slices of a per-epoch permutation of the training set."""
    dev = data.feat.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed) + 17)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    per_epoch = max(1, data.count // batch)
    hist = []
    feat, lab = data.feat, data.label
    for step in range(int(steps)):
        k = step % per_epoch
        if k == 0:
            perm = torch.randperm(data.count, generator=gen, device=dev)
            feat = data.feat.index_select(0, perm)
            lab = data.label.index_select(0, perm)
        lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / max(1, steps)))
        mlp.train_step(feat[k * batch:(k + 1) * batch], lab[k * batch:(k + 1) * batch], lr, loss)
        if log_every and (step % log_every == 0 or step == steps - 1):
            rec = {"step": step, "lr": lr, "loss": float(loss.item())}
            if val is not None:
                rec.update(evaluate(mlp, val))
            hist.append(rec)
            if callback:
                callback(rec)
    return hist


def add_hardest(mlp: "spl.Mlp", data: FootprintSet, pool: FootprintSet, count: int, copies: int = 2):
    """Append to the training set the `count` samples of `pool` on which
    f_theta (as the tensor-core kernel evaluates it) errs most, `copies`
    times each (hard-example mining: more weight where the network is
    worst)."""
    out = torch.empty_like(pool.label)
    spl.footprint(spl.basis(pool.degree, spl.SPL_FP_MLP, mlp), pool.omega, pool.p, out)
    idx = torch.topk((out - pool.label).abs(), min(int(count), pool.count)).indices
    data.feat = torch.cat([data.feat] + [pool.feat.index_select(0, idx)] * copies)
    data.label = torch.cat([data.label] + [pool.label.index_select(0, idx)] * copies)
    data.count = int(data.label.numel())


# The training recipe of the measurements: Algorithm 1's samples kept inside
# the exact support, half of the directions near the coordinate axes and
# offsets drawn toward the peak; 200 000 Adam steps, then two rounds of
# hard-example mining (the 2^19 worst of 2^23 fresh in-support samples added
# twice, 150 000 more steps each).
RECIPE = {"set": dict(support_only=True, axis_fraction=0.5, axis_scale=12.0, center_power=3.0),
          "steps": 200000, "lr0": 3e-3, "lr_min": 1e-5, "mine_rounds": 2, "mine_pool": 1 << 23,
          "mine_count": 1 << 19, "mine_steps": 150000, "mine_lr0": 1e-3}


def train_recipe(mlp: "spl.Mlp", degree: int, count: int = 1 << 22, seed: int = 31, scale: float = 1.0,
                 device="cuda") -> FootprintSet:
    """Train f_theta with RECIPE (step counts times `scale`); returns the
    final training set."""
    r = RECIPE
    data = FootprintSet(degree, count, seed=seed, device=device, **r["set"])
    train(mlp, data, steps=max(1, int(r["steps"] * scale)), batch=8192, lr0=r["lr0"], lr_min=r["lr_min"])
    for k in range(r["mine_rounds"]):
        pool = FootprintSet(degree, r["mine_pool"], seed=seed + 1000 + k, device=device, support_only=True)
        add_hardest(mlp, data, pool, r["mine_count"])
        del pool
        train(mlp, data, steps=max(1, int(r["mine_steps"] * scale)), batch=8192, lr0=r["mine_lr0"], lr_min=1e-6,
              seed=k + 1)
    return data


def save(mlp: "spl.Mlp", path: str):
    """Checkpoint of the training state (spl_mlp_save: header with the
    network's shape, degree, dtype, seed and Adam step; master parameters and
    Adam moments)."""
    mlp.save(path)


def load(mlp: "spl.Mlp", path: str):
    """Restore a checkpoint written by save (spl_mlp_load); training resumes
    where it stopped."""
    mlp.load(path)
