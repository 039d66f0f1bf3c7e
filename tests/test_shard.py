"""View-sharded operators and CGLS across ranks, on CPU with gloo.

Two ranks each own a block of the views; their operators here are the FP64
oracle's (test infrastructure), so the test checks the sharding logic of
paper_2511_11078_gb300.shard exactly: the sharded forward concatenates to
the full forward, the all-reduced partial adjoints sum to the full adjoint,
and five sharded CGLS iterates equal the single-rank FP64 CGLS iterates.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DIMS = (9, 8, 7)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _geometry():
    from paper_2511_11078_gb300 import inputs as I

    return I.helical_cone(7, 30.0, 45.0, 9, 8, 1.3, turns=0.6, table_feed=3.0)


def _oracle_geom(orc, geo):
    return orc.Geometry("cone", source=geo.src, det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v,
                        nu=geo.nu, nv=geo.nv)


class OracleOps:
    """ShardOps on one rank's block of views with the FP64 oracle (torch
    float64 CPU tensors in and out)."""

    def __init__(self, orc, geo, v0, v1, degree=3):
        import torch

        from paper_2511_11078_gb300 import inputs as I

        self.t = torch
        self.orc = orc
        self.n = degree
        self.origin = I.centred_origin(DIMS)
        self.g = _oracle_geom(orc, geo.subset_views(np.arange(v0, v1)))

    def forward(self, c, out):
        out.copy_(self.t.from_numpy(self.orc.forward(self.n, DIMS, self.origin, c.numpy(), self.g)))

    def adjoint(self, y, out):
        out.copy_(self.t.from_numpy(self.orc.adjoint(self.n, DIMS, self.origin, y.numpy(), self.g)))

    def dot(self, a, b, out):
        out[0] = float(np.dot(a.numpy().ravel(), b.numpy().ravel()))

    def step_x(self, x, p, r, q, num, den):
        alpha = float(num[0]) / float(den[0]) if float(den[0]) != 0.0 else 0.0
        x.add_(alpha * p)
        r.sub_(alpha * q)

    def step_p(self, p, s, num, den):
        beta = float(num[0]) / float(den[0]) if float(den[0]) != 0.0 else 0.0
        p.mul_(beta).add_(s)


def _worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import oracle

    from paper_2511_11078_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    geo = _geometry()
    v0, v1 = shard.view_blocks(geo.n_views, ws)[rank]
    ops = OracleOps(oracle, geo, v0, v1)
    rng = np.random.default_rng(77)
    c = torch.from_numpy(rng.normal(size=DIMS[::-1]))
    y = torch.from_numpy(rng.normal(size=geo.n_rays))
    rows = slice(v0 * geo.nu * geo.nv, v1 * geo.nu * geo.nv)
    yl = torch.empty(v1 * geo.nu * geo.nv - v0 * geo.nu * geo.nv, dtype=torch.float64)
    ops.forward(c, yl)
    ct = torch.empty_like(c)
    ops.adjoint(y[rows].clone(), ct)
    shard.allreduce_sum(ct)
    cg = shard.ShardedCGLS(ops, y[rows].clone(), c.shape)
    xs = []
    for _ in range(5):
        cg.step()
        xs.append(cg.x.numpy().copy())
    out.put((rank, (v0, v1), yl.numpy(), ct.numpy(), xs))
    dist.barrier()
    dist.destroy_process_group()


def test_view_blocks_partition_the_views():
    sys.path.insert(0, ROOT)
    from paper_2511_11078_gb300 import shard

    for n, w in [(720, 1), (720, 8), (7, 2), (5, 8), (0, 3)]:
        b = shard.view_blocks(n, w)
        assert len(b) == w and b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(w - 1))
        sizes = [v1 - v0 for v0, v1 in b]
        assert max(sizes) - min(sizes) <= 1


def test_sharded_operators_and_cgls_with_two_gloo_ranks(orc):
    import torch.multiprocessing as mp

    from oracle import cgls as ocg
    from paper_2511_11078_gb300 import inputs as I

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    geo = _geometry()
    origin = I.centred_origin(DIMS)
    og = _oracle_geom(orc, geo)
    rng = np.random.default_rng(77)
    c = rng.normal(size=DIMS[::-1])
    y = rng.normal(size=geo.n_rays)
    # forward: the ranks' rows concatenate to the full forward
    full = orc.forward(3, DIMS, origin, c, og)
    np.testing.assert_allclose(np.concatenate([r[2] for r in res]), full, rtol=1e-13, atol=1e-13)
    # adjoint: the all-reduced partials equal the full adjoint on every rank
    ref = orc.adjoint(3, DIMS, origin, y, og)
    for r in res:
        np.testing.assert_allclose(r[3], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # CGLS: both ranks hold the single-rank FP64 iterates
    xs_ref, _ = ocg.cgls(lambda v: orc.forward(3, DIMS, origin, v, og), lambda v: orc.adjoint(3, DIMS, origin, v, og),
                         y, 5)
    for r in res:
        for k in range(5):
            np.testing.assert_allclose(r[4][k], xs_ref[k], rtol=0, atol=1e-10 * np.abs(xs_ref[k]).max())
    np.testing.assert_array_equal(res[0][4][-1], res[1][4][-1])
