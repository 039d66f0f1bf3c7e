"""View-sharded A, A^T and CGLS with the library's kernels: two ranks (two
processes sharing one GPU, gloo collectives on host-staged copies; no kernel
waits on another) against the single-rank results of the same operators.
The kernels of the two processes are independent launches: the only
exchange is the host-side all-reduce between them."""
import os
import socket
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (40, 38, 36)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    from paper_2511_11078_gb300 import inputs as I

    geo = I.helical_cone(24, 120.0, 180.0, 33, 29, 2.0, turns=1.2, table_feed=6.0)
    rng = np.random.default_rng(88)
    c = rng.normal(size=DIMS[::-1]).astype(np.float32)
    y = rng.normal(size=geo.n_rays).astype(np.float32)
    return geo, c, y


def _worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import shard, spl

    torch.cuda.set_device(0)
    spl.lib()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    geo, c, y = _workload()
    ops = shard.ShardedProjector(DIMS, I.centred_origin(DIMS), geo, rank, ws)
    ct = torch.tensor(c, device="cuda")
    yl = torch.tensor(y[ops.rows], device="cuda")
    yf = torch.empty_like(yl)
    ops.forward(ct, yf)
    cb = torch.empty_like(ct)
    ops.adjoint(yl, cb)
    shard.allreduce_sum(cb, host_staged=True)
    cg = shard.ShardedCGLS(ops, yl, ct.shape, host_staged=True)
    xs = []
    for _ in range(5):
        cg.step()
        xs.append(cg.x.cpu().numpy().copy())
    torch.cuda.synchronize()
    ops.geom.status()
    out.put((rank, yf.cpu().numpy(), cb.cpu().numpy(), xs))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_operators_and_cgls_on_two_ranks():
    import torch
    import torch.multiprocessing as mp

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import spl
    from paper_2511_11078_gb300.recon import CGLS, Projector

    B.build()
    spl.lib()
    geo, c, y = _workload()
    # single rank, the same kernels (taken before the workers start)
    g = spl.Geometry(DIMS, I.centred_origin(DIMS), geo)
    proj = Projector(g, 3)
    ct = torch.tensor(c, device="cuda")
    yt = torch.tensor(y, device="cuda")
    yref = proj.forward(ct).cpu().numpy().reshape(-1)
    cref = proj.adjoint(yt).cpu().numpy()
    cg = CGLS(proj, yt)
    xs_ref = []
    for _ in range(5):
        cg.step()
        xs_ref.append(cg.x.cpu().numpy().copy())
    torch.cuda.synchronize()
    g.status()

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0

    def rel(a, b):
        return np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b)

    assert rel(np.concatenate([r[1] for r in res]), yref) <= 1e-6
    for r in res:
        assert rel(r[2], cref) <= 1e-6
        for k in range(5):
            assert rel(r[3][k], xs_ref[k]) <= 1e-6, (k, rel(r[3][k], xs_ref[k]))
    np.testing.assert_array_equal(res[0][3][-1], res[1][3][-1])
