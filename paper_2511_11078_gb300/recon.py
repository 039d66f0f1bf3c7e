"""Operators, autograd and least-squares reconstruction on top of libspl.so.

* ``Projector``      -- A (spl_forward) and A^T (spl_adjoint) on CUDA tensors.
* ``SplineXray``     -- torch.autograd.Function: forward A c, backward A^T g.
* ``SplineXrayT``    -- torch.autograd.Function: forward A^T y, backward A g.
* ``cgls``           -- conjugate gradients on the normal equations of the
                        least-squares problem of Eq. 5 (no regularisation,
                        x0 = 0), FP64 inner products on the GPU (spl_dot_f64)
                        and device-side step sizes (no host sync per step).

PyTorch provides memory and streams only: every arithmetic step of the
operators, the inner products and the CG updates runs in the library's
kernels.
"""
from __future__ import annotations

import torch

from . import spl


class Projector:
    """A and A^T for one geometry and basis (degree, footprint mode)."""

    def __init__(self, geometry: "spl.Geometry", degree: int = 3, mode: int = spl.SPL_FP_QUAD, mlp=None,
                 kahan: bool = True):
        self.geometry = geometry
        self.degree = int(degree)
        self.mode = int(mode)
        self.mlp = mlp
        self.basis = spl.basis(degree, mode, mlp, kahan)

    @property
    def coeff_shape(self):
        return self.geometry.coeff_shape

    @property
    def proj_shape(self):
        return self.geometry.shape

    def forward(self, c: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        c = c.contiguous()
        if out is None:
            out = torch.empty(self.proj_shape, dtype=torch.float32, device=c.device)
        spl.forward(self.geometry, c, out, self.basis)
        return out

    def adjoint(self, y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        y = y.contiguous()
        if out is None:
            out = torch.empty(self.coeff_shape, dtype=torch.float32, device=y.device)
        spl.adjoint(self.geometry, y, out, self.basis)
        return out


class SplineXray(torch.autograd.Function):
    """y = A c with dL/dc = A^T dL/dy (the matched adjoint kernel)."""

    @staticmethod
    def forward(ctx, c, proj: Projector):
        ctx.proj = proj
        return proj.forward(c)

    @staticmethod
    def backward(ctx, g):
        return ctx.proj.adjoint(g), None


class SplineXrayT(torch.autograd.Function):
    """c = A^T y with dL/dy = A dL/dc."""

    @staticmethod
    def forward(ctx, y, proj: Projector):
        ctx.proj = proj
        return proj.adjoint(y)

    @staticmethod
    def backward(ctx, g):
        return ctx.proj.forward(g), None


def project(c: torch.Tensor, proj: Projector) -> torch.Tensor:
    return SplineXray.apply(c, proj)


def backproject(y: torch.Tensor, proj: Projector) -> torch.Tensor:
    return SplineXrayT.apply(y, proj)


class CGLS:
    """Conjugate gradients for min ||A x - y||^2 (Eq. 5) on the normal
    equations A^T A x = A^T y, x0 = 0, without preconditioner or
    regularisation:

        r = y, s = A^T r, p = s, gamma = <s, s>
        repeat:  q = A p;  alpha = gamma / <q, q>
                 x += alpha p;  r -= alpha q
                 s = A^T r;  gamma' = <s, s>;  p = s + (gamma'/gamma) p

    One iteration = one A, one A^T, two FP64 inner products and two fused
    vector updates, all on the GPU; the FP64 scalars stay on the device.
    """

    def __init__(self, proj: Projector, y: torch.Tensor, x0: torch.Tensor | None = None):
        self.A = proj
        dev = y.device
        self.y = y.contiguous()
        self.x = torch.zeros(proj.coeff_shape, dtype=torch.float32, device=dev) if x0 is None else x0.clone()
        self.r = self.y.clone()
        if x0 is not None:
            self.r -= proj.forward(self.x)
        self.q = torch.empty_like(self.y)
        self.s = proj.adjoint(self.r)
        self.p = self.s.clone()
        self.work = spl.dot_workspace(dev)
        self.gamma = torch.zeros(1, dtype=torch.float64, device=dev)
        self.gamma_new = torch.zeros(1, dtype=torch.float64, device=dev)
        self.qq = torch.zeros(1, dtype=torch.float64, device=dev)
        spl.dot_f64(self.s, self.s, self.gamma, self.work)
        self.iterations = 0

    def step(self):
        A = self.A
        A.forward(self.p, out=self.q)
        spl.dot_f64(self.q, self.q, self.qq, self.work)
        spl.cg_step_x(self.x, self.p, self.r, self.q, self.gamma, self.qq)
        A.adjoint(self.r, out=self.s)
        spl.dot_f64(self.s, self.s, self.gamma_new, self.work)
        spl.cg_step_p(self.p, self.s, self.gamma_new, self.gamma)
        self.gamma, self.gamma_new = self.gamma_new, self.gamma
        self.iterations += 1

    def residual_norm(self) -> float:
        out = torch.zeros(1, dtype=torch.float64, device=self.y.device)
        spl.dot_f64(self.r, self.r, out, self.work)
        return float(out.sqrt().item())

    def run(self, iters: int, callback=None):
        for _ in range(int(iters)):
            self.step()
            if callback is not None:
                callback(self)
        return self.x


def cgls(proj: Projector, y: torch.Tensor, iters: int, callback=None) -> torch.Tensor:
    return CGLS(proj, y).run(iters, callback)
