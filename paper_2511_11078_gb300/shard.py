"""View-sharded operators and least squares across ranks (one GPU each).

The rows of the system matrix of Eq. 6 are the rays, and the rays of a view
geometry group by view; so the views split across ranks with no change to
any row:

* A (forward): rank r projects its own block of views into its own block of
  y; no exchange.
* A^T (adjoint): every rank backprojects its block of y into a full-size
  partial c; one sum over ranks (all-reduce) gives A^T y.
* CGLS (Eq. 5 on the normal equations): x, p and s = A^T r are replicated
  (identical on every rank: s comes out of the all-reduce, and the updates
  are deterministic), r and q = A p are sharded like y; the FP64 inner
  product <q, q> is a sum over ranks of the shards' inner products (one
  scalar all-reduce), <s, s> is computed locally on the replicated s.

The operators are callables, so the same sharding logic runs with the
library's GPU kernels (ShardedProjector) and, in the tests, with any other
implementation of A and A^T.  The collective is torch.distributed's
all_reduce (NCCL between GPUs; gloo on host-staged copies where NCCL is not
available).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def view_blocks(n_views: int, world: int):
    """Contiguous blocks of views, one per rank, sizes differing by at most
    one: [(v0, v1) for rank 0 .. world-1]."""
    base, extra = divmod(int(n_views), int(world))
    out, v = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((v, v + n))
        v += n
    return out


def allreduce_sum(t: torch.Tensor, host_staged: bool = False) -> torch.Tensor:
    """In-place sum over ranks.  host_staged: copy to host memory for the
    collective (gloo with CUDA tensors) and back."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return t
    if host_staged and t.is_cuda:
        h = t.cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


class ShardOps:
    """The three operations CGLS needs on one rank's shard: forward (c ->
    this rank's rows of y), adjoint (this rank's rows of y -> partial c),
    dot (FP64 inner product of two local vectors, returned as a 1-element
    FP64 tensor), and the two CG updates."""

    def forward(self, c, out):
        raise NotImplementedError

    def adjoint(self, y, out):
        raise NotImplementedError

    def dot(self, a, b, out):
        raise NotImplementedError

    def step_x(self, x, p, r, q, num, den):
        raise NotImplementedError

    def step_p(self, p, s, num, den):
        raise NotImplementedError


class ShardedCGLS:
    """CGLS for min ||A x - y||^2 with A sharded by views (see the module
    docstring).  y_local: this rank's rows of y.  With one rank it is plain
    CGLS (the same algorithm as recon.CGLS)."""

    def __init__(self, ops: ShardOps, y_local, coeff_shape, host_staged: bool = False):
        self.ops = ops
        self.hs = host_staged
        like = y_local
        self.r = y_local.clone()
        self.q = torch.empty_like(y_local)
        self.x = torch.zeros(coeff_shape, dtype=like.dtype, device=like.device)
        self.s = torch.empty(coeff_shape, dtype=like.dtype, device=like.device)
        self.ops.adjoint(self.r, self.s)
        allreduce_sum(self.s, self.hs)
        self.p = self.s.clone()
        dev = like.device
        self.gamma = torch.zeros(1, dtype=torch.float64, device=dev)
        self.gamma_new = torch.zeros(1, dtype=torch.float64, device=dev)
        self.qq = torch.zeros(1, dtype=torch.float64, device=dev)
        self.ops.dot(self.s, self.s, self.gamma)
        self.iterations = 0

    def step(self, mark=None):
        """One iteration.  mark (optional) is called with 0 .. 4 at the
        iteration's start, after A, before A^T, after A^T and at its end
        (a benchmark records CUDA events there)."""
        ops = self.ops
        mark = mark or (lambda i: None)
        mark(0)
        ops.forward(self.p, self.q)                       # A p: this rank's rows, no exchange
        mark(1)
        ops.dot(self.q, self.q, self.qq)
        allreduce_sum(self.qq, self.hs)                   # <q, q> over all rows
        ops.step_x(self.x, self.p, self.r, self.q, self.gamma, self.qq)
        mark(2)
        ops.adjoint(self.r, self.s)                       # this rank's part of A^T r
        mark(3)
        allreduce_sum(self.s, self.hs)                    # A^T r (the one N^3 exchange)
        ops.dot(self.s, self.s, self.gamma_new)           # s replicated: local
        ops.step_p(self.p, self.s, self.gamma_new, self.gamma)
        self.gamma, self.gamma_new = self.gamma_new, self.gamma
        self.iterations += 1
        mark(4)

    def run(self, iters: int):
        for _ in range(int(iters)):
            self.step()
        return self.x


class ShardedProjector(ShardOps):
    """The library's operators on one rank's block of views of a view
    geometry (inputs.ViewGeometry): spl_forward / spl_adjoint on the
    sub-geometry of those views, spl_dot_f64 and the CG updates."""

    def __init__(self, dims, origin, geometry, rank: int, world: int, degree: int = 3, basis=None):
        from . import spl

        self.spl = spl
        self.v0, self.v1 = view_blocks(geometry.n_views, world)[rank]
        self.views = np.arange(self.v0, self.v1)
        self.geom = spl.Geometry(dims, origin, geometry.subset_views(self.views))
        self.basis = basis if basis is not None else spl.basis(degree)
        self.work = spl.dot_workspace()
        self.rows = slice(self.v0 * geometry.nu * geometry.nv, self.v1 * geometry.nu * geometry.nv)

    def forward(self, c, out):
        self.spl.forward(self.geom, c, out, self.basis)

    def adjoint(self, y, out):
        self.spl.adjoint(self.geom, y, out, self.basis)

    def dot(self, a, b, out):
        self.spl.dot_f64(a, b, out, self.work)

    def step_x(self, x, p, r, q, num, den):
        self.spl.cg_step_x(x, p, r, q, num, den)

    def step_p(self, p, s, num, den):
        self.spl.cg_step_p(p, s, num, den)
