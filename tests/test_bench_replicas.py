"""The benchmark's multi-process bookkeeping on CPU (gloo, world size 2): the
step time is the maximum over ranks, the value is the whole job's
contributions over that time, and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.max_over_ranks(times[rank], ws)
    out.put((rank, ms, bench.job_value(2e9, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 20.0  # the slowest rank's step time on every rank
        assert value == pytest.approx(2e9 / 20e-3 / 1e9)  # the whole job's work over that time


def test_one_rank_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_value(2e9, 10.0) == pytest.approx(200.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under a launcher, ranks other than 0 exit at once without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_stratified_ray_sample_covers_the_classes():
    """The oracle leg's ray sample: seeded, unique, in range, at least the
    requested size, and holding detector edge rows and columns, the first
    and last views."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2511_11078_gb300 import inputs as I

    geo = I.helical_cone(720, 1000.0, 1500.0, 768, 768, 0.8, turns=2.0, table_feed=204.8)
    r = bench.stratified_rays(geo, 4096, seed=2026)
    assert np.array_equal(r, bench.stratified_rays(geo, 4096, seed=2026))
    assert r.size >= 4096 * 0.98 and np.unique(r).size == r.size
    assert r.min() >= 0 and r.max() < geo.n_rays
    view, rem = np.divmod(r, geo.nu * geo.nv)
    iv, iu = np.divmod(rem, geo.nu)
    assert np.any(view == 0) and np.any(view == geo.n_views - 1)
    for edge in (iu == 0, iu == geo.nu - 1, iv == 0, iv == geo.nv - 1):
        assert np.count_nonzero(edge) >= 50


def test_ncu_traffic_only_for_current_sources(tmp_path, monkeypatch):
    """A kernel's DRAM traffic is taken from a committed ncu summary only
    while the CUDA sources hash to the value the summary names."""
    sys.path.insert(0, ROOT)
    import bench

    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = bench.csrc_sha16()
    (prof / "k.md").write_text("x\ntraffic_bytes_per_launch k_foo wl-a 1.5e9 csrc %s\n"
                               "traffic_bytes_per_launch k_bar wl-a 2.5e9 csrc 0123456789abcdef\n" % sha)
    real_glob = bench.glob.glob
    monkeypatch.setattr(bench.glob, "glob", lambda pat: real_glob(str(prof / "*.md")) if "profiles" in pat
                        else real_glob(pat))
    assert bench.ncu_traffic("k_foo", "wl-a") == 1.5e9
    assert bench.ncu_traffic("k_foo", "wl-b") is None
    assert bench.ncu_traffic("k_bar", "wl-a") is None  # stale: another source hash


def test_launch_count_follows_the_adjoint_batches():
    """The claimed kernel launches per CGLS iteration: A, two dots of two
    kernels, two updates, and A^T as scatter + two layout folds per batch of
    48 views, with the FP64 batch totals and final rounding once batched."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.launches_per_cg_step(48) == 1 + 4 + 2 + 3
    assert bench.launches_per_cg_step(49) == 1 + 4 + 2 + 2 * 4 + 1
    assert bench.launches_per_cg_step(720) == 1 + 4 + 2 + 15 * 4 + 1
    assert bench.launches_per_cg_step(720, scatter=False) == 8
