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
    """`count` exact-footprint samples of Algorithm 1 resident on the GPU."""

    def __init__(self, degree: int, count: int, seed: int, device="cuda"):
        self.degree = int(degree)
        gen = torch.Generator(device=device)
        gen.manual_seed(int(seed))
        normals = torch.randn((count, 3), generator=gen, device=device)
        uniforms = torch.rand((count, 2), generator=gen, device=device)
        self.omega = torch.empty((count, 3), dtype=torch.float32, device=device)
        self.p = torch.empty((count, 3), dtype=torch.float32, device=device)
        spl.footprint_samples(degree, normals, uniforms, self.omega, self.p)
        self.feat = torch.empty((count, 5), dtype=torch.float32, device=device)
        spl.features(degree, self.omega, self.p, self.feat)
        self.label = torch.empty(count, dtype=torch.float32, device=device)
        spl.footprint(spl.basis(degree), self.omega, self.p, self.label)
        self.count = count

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


def save(mlp: "spl.Mlp", path: str):
    """Checkpoint of the training state (spl_mlp_save: header with the
    network's shape, degree, dtype, seed and Adam step; master parameters and
    Adam moments)."""
    mlp.save(path)


def load(mlp: "spl.Mlp", path: str):
    """Restore a checkpoint written by save (spl_mlp_load); training resumes
    where it stopped."""
    mlp.load(path)
