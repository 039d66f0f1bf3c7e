#!/usr/bin/env python3
"""Benchmark of the B-spline x-ray transform (SplineSplat, arXiv 2511.11078).

Workload (one GPU): 128^3 FP32 cubic B-spline coefficients of a 6-ellipsoid
phantom, parallel beam, 180 single-axis tilt views over [0, 180 deg) plus 64
random directions, 192x192 detector, pitch 1; data y = A c_true + Gaussian
noise (sigma = 1% of max).  One step = one CGLS iteration of the
least-squares problem of Eq. 5: one forward projection A, one matched
adjoint A^T, two FP64 inner products and the two CG vector updates, all on
the GPU with the exact quadrature footprint.  The 180 tilt views are
slice-separable (flat rays, detector rows along e3) and go through the plane
matrices (built once, outside the timed region); the 64 random views through
the cell march.  view_classes reports A and A^T of each class alone.

Metric: contributions (ray, basis pairs of Eq. 4) processed per second by
A and A^T, in G-contributions/s; also seconds per reconstruction iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (as it stands) on the host cores,
each step a bounded sample of the same workload.  Under torchrun (N > 1)
every rank runs an independent replica of the workload on its own GPU
(weak scaling; the operators need no exchange between replicas); rank 0
prints the JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "A/A^T G-contributions/s (exact quadrature footprint, one CGLS iteration per step)"
UNIT = "Gcontrib/s"
WORKLOAD = "tilt-128^3-cubic-parallel-244x192^2"

# FP32 arithmetic per Gauss node of the cell march (node position, two
# transverse arguments, three sets of n+1 B-spline weights, node weight,
# d-weight scaling, (n+1)^2 transverse products, (n+1)^3 FMAs) and per flushed
# contribution (one FMA).
FLOP_PER_NODE = {0: 11, 1: 32, 2: 94, 3: 200}
# flat rays (a zero direction component): n+1 nodes per piece, no b-weights,
# an (n+1)^2 update per node
FLOP_PER_FLAT_NODE = {0: 8, 1: 17, 2: 40, 3: 71}
MLP_FLOP_PER_PAIR = 2 * (5 * 64 + 2 * 64 * 64 + 64)
FLOP_PER_PAIR = 2
NODES_PER_PIECE = {0: 1, 1: 2, 2: 4, 3: 5}
SMS, FP32_LANES = 152, 128
# DRAM bytes (read + write) per launch from the ncu capture of each kernel
# on this workload (profiles/k_*_pviews*-general-tilt128-cubic.md: the general-view
# launches); to be reset to None
# whenever the kernel changes after the capture.
NCU_TRAFFIC = {"k_forward_pviews": 8.487168e6 + 1024.0, "k_adjoint_pviews_scatter": 17.908736e6 + 768.0,
               "k_adjoint_bricks": None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--adjoint", default="scatter", choices=["gather", "scatter"],
                    help="form of A^T: ray-driven scatter (float atomics, the library default) or brick gather")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mlp-steps", type=int, default=200000,
                    help="Adam steps of the learned footprint trained before the MLP measurement (0: skip it)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target seconds of the CPU-baseline sample")
    ap.add_argument("--mlp-views", default=None, metavar="START:STOP",
                    help="only run the learned-footprint projector (f_theta seeded 5, trained for --mlp-steps "
                         "steps first) once forward and once adjoint on views START..STOP-1 of the workload and "
                         "print their times (a small case for profiling)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """The largest of the ranks' values (the step time of the slowest
    replica); the value itself at one rank."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ws: int, contributions_per_step: float, ms: float) -> float:
    """Whole-job throughput of ws independent replicas (weak scaling): the
    contributions all ranks processed per second at the slowest rank's step
    time, in G-contributions/s."""
    return ws * contributions_per_step / (ms * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread is not None:
                self.thread.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            t = [x.strip() for x in ln.split(",")]
            if len(t) < 8:
                continue
            try:
                sm.append(float(t[0]))
                smax.append(float(t[1]))
            except ValueError:
                continue
            for name, v in zip(names, t[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded ray sample of the workload
# --------------------------------------------------------------------------
def oracle_geometry(oracle, geo):
    return oracle.Geometry("parallel", direction=geo.src, det_center=geo.det_center, det_u=geo.det_u,
                           det_v=geo.det_v, nu=geo.nu, nv=geo.nv)


def oracle_step(oracle, wl, og, rays, y_sample, threads):
    """Oracle A on the sampled rays and A^T of y restricted to them; returns
    (seconds, contributions of A + A^T)."""
    t0 = time.perf_counter()
    _, pairs = oracle.forward_subset(wl.degree, wl.dims, wl.origin, wl.coeffs, og, rays, nthreads=threads)
    _, pairs_t = oracle.adjoint_subset(wl.degree, wl.dims, wl.origin, y_sample, og, rays, nthreads=threads)
    return time.perf_counter() - t0, int(pairs.sum()) + int(pairs_t)


def oracle_sample(oracle, wl, og, seconds, threads, seed=11):
    """Ray sample sized so one oracle step (A + A^T) takes about `seconds`."""
    rng = np.random.default_rng(seed)
    n_rays = wl.geometry.n_rays
    probe = np.sort(rng.choice(n_rays, 256, replace=False))
    t, _ = oracle_step(oracle, wl, og, probe, np.ones(probe.size), threads)
    count = int(min(n_rays, max(256, 256 * seconds / max(t, 1e-3))))
    rays = np.sort(rng.choice(n_rays, count, replace=False))
    return rays, rng.uniform(0, 1, count)


def cpu_baseline(wl, seconds):
    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    og = oracle_geometry(oracle, wl.geometry)
    rays, ys = oracle_sample(oracle, wl, og, seconds, threads)
    t, pairs = oracle_step(oracle, wl, og, rays, ys, threads)
    return {"value": pairs / t / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of %d rays (seeded uniform sample) of the %s workload: oracle A on them plus A^T of a "
                      "random y on them; %.1f s" % (rays.size, wl.geometry.n_rays, WORKLOAD, t)}


# --------------------------------------------------------------------------
# reference arm: the oracle timed as the benchmark step
# --------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2511_11078_gb300 import inputs as I

    oracle.build()
    threads = os.cpu_count() or 1
    wl = I.workload_tilt(args.degree)
    wl.coeffs = wl.coeffs.astype(np.float64)
    og = oracle_geometry(oracle, wl.geometry)
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    rays, ys = oracle_sample(oracle, wl, og, per_step, threads)
    for _ in range(args.warmup):
        oracle_step(oracle, wl, og, rays, ys, threads)
    tt, pp = 0.0, 0
    for _ in range(args.steps):
        t, p = oracle_step(oracle, wl, og, rays, ys, threads)
        tt += t
        pp += p
    value = pp / tt / 1e9
    sample = "%d of %d rays (seeded uniform sample) per step: oracle A on them plus A^T of a random y on them" % (
        rays.size, wl.geometry.n_rays)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "degree": args.degree, "footprint": "exact quadrature (FP64)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# learned footprint: train f_theta (Algorithm 1), then time A and A^T with it
# --------------------------------------------------------------------------
def mlp_measure(args, wl, geom, c_true, y, pairs, proj, dev):
    import torch

    from paper_2511_11078_gb300 import learn, spl

    n = args.degree
    t0 = time.perf_counter()
    data = learn.FootprintSet(n, 1 << 22, seed=31, device=dev)
    val = learn.FootprintSet(n, 1 << 16, seed=32, device=dev)
    mlp = spl.Mlp(n, max_batch=8192, seed=5)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    learn.train(mlp, data, steps=args.mlp_steps, batch=8192, lr0=3e-3, lr_min=1e-6)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    acc = learn.evaluate(mlp, val)
    b = spl.basis(n, spl.SPL_FP_MLP, mlp)
    yq = torch.empty_like(y)
    ym = torch.empty_like(y)
    cm = torch.empty_like(c_true)
    cq = torch.empty_like(c_true)
    proj.forward(c_true, out=yq)
    spl.forward(geom, c_true, ym, b)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    spl.forward(geom, c_true, ym, b)
    ev[1].record(stream)
    spl.adjoint(geom, y, cm, b)
    ev[2].record(stream)
    torch.cuda.synchronize()
    geom.status()
    a_ms, at_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    proj.adjoint(y, out=cq)
    torch.cuda.synchronize()
    return {"footprint": "f_theta 5-64-64-64-1 SiLU, BF16 weights/activations, FP32 accumulation (tcgen05, accumulator in TMEM)",
            "A_ms": a_ms, "AT_ms": at_ms, "A_gcontrib_s": pairs / a_ms / 1e6, "AT_gcontrib_s": pairs / at_ms / 1e6,
            "s_per_recon_iter_est": (a_ms + at_ms) / 1e3,
            "tensor_tflops_A": pairs * MLP_FLOP_PER_PAIR / a_ms / 1e9,
            "train_steps": args.mlp_steps, "train_batch": 8192, "train_samples": 1 << 22,
            "train_s": t2 - t1, "dataset_s": t1 - t0,
            "footprint_max_abs_over_peak": acc["max_abs_rel_peak"], "footprint_rms": acc["rms"],
            "A_rel_l2_vs_exact": float((ym - yq).norm() / yq.norm()),
            "AT_rel_l2_vs_exact": float((cm - cq).norm() / cq.norm())}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import spl
    from paper_2511_11078_gb300.recon import CGLS, Projector

    B.build()
    spl.lib()
    n = args.degree
    wl = I.workload_tilt(n)
    geom = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    form = spl.SPL_ADJ_GATHER if args.adjoint == "gather" else spl.SPL_ADJ_SCATTER
    proj = Projector(geom, n)
    proj.basis = spl.basis(n, adjoint=form)
    c_true = torch.tensor(wl.coeffs, device=dev)
    y_clean = proj.forward(c_true)
    gen = torch.Generator(device=dev)
    gen.manual_seed(I.SEED_BASE + 2)
    sigma = 0.01 * float(y_clean.max())
    y = y_clean + sigma * torch.randn(y_clean.shape, generator=gen, device=dev)
    pairs, pieces, flat_pieces = spl.count_work(geom, n)
    geom.status()
    # one-time plane-matrix build of the slice-separable views (outside the
    # timed region; the first forward above already did it, this reads the
    # cost on a fresh geometry)
    g_fresh = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    torch.cuda.synchronize()
    t_build = time.perf_counter()
    spl.prepare(g_fresh, proj.basis)
    torch.cuda.synchronize()
    plane_build_s = time.perf_counter() - t_build
    del g_fresh
    # view classes: slice-separable (plane matrices) and general (cell march)
    src = np.asarray(wl.geometry.src)
    flat = np.any(src == 0.0, axis=1)
    classes = {}
    for name, views in (("separable", np.nonzero(flat)[0]), ("general", np.nonzero(~flat)[0])):
        if len(views) == 0:
            continue
        gsub = spl.Geometry(wl.dims, wl.origin, wl.geometry.subset_views(views))
        p_, pc_, pf_ = spl.count_work(gsub, n)
        classes[name] = {"views": int(len(views)), "geom": gsub, "pairs": p_, "pieces": pc_, "flat_pieces": pf_}

    cg = CGLS(proj, y)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def l2_flush():
        flush.fill_(1.0)

    for _ in range(args.warmup):
        cg.step()
    torch.cuda.synchronize()
    geom.status()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local]))
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        l2_flush()
        e0, e1, e2 = ev[k]
        e0.record(stream)
        proj.forward(cg.p, out=cg.q)          # A (timed separately below)
        e1.record(stream)
        spl.dot_f64(cg.q, cg.q, cg.qq, cg.work)
        spl.cg_step_x(cg.x, cg.p, cg.r, cg.q, cg.gamma, cg.qq)
        proj.adjoint(cg.r, out=cg.s)
        spl.dot_f64(cg.s, cg.s, cg.gamma_new, cg.work)
        spl.cg_step_p(cg.p, cg.s, cg.gamma_new, cg.gamma)
        cg.gamma, cg.gamma_new = cg.gamma_new, cg.gamma
        e2.record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        torch.distributed.barrier()
    sampler.stop()
    geom.status()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    fwd_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    ms = max_over_ranks(sum(step_ms) / args.steps, ws, dev)

    # adjoint alone (events around one launch, after an L2 flush)
    adj_ms = []
    for _ in range(3):
        l2_flush()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        proj.adjoint(cg.r, out=cg.s)
        a1.record(stream)
        torch.cuda.synchronize()
        adj_ms.append(a0.elapsed_time(a1))
    fwd = statistics.median(fwd_ms)
    adj = statistics.median(adj_ms)

    # per view class: A and A^T of the class alone (the same kernels and launch
    # shapes as inside the step), events around each call after an L2 flush
    def time_call(fn, reps=3):
        out = []
        for _ in range(reps):
            l2_flush()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            fn()
            t1.record(stream)
            torch.cuda.synchronize()
            out.append(t0.elapsed_time(t1))
        return statistics.median(out)

    per_class = {}
    for name, cl in classes.items():
        gsub = cl["geom"]
        ysub = torch.empty(gsub.n_rays, dtype=torch.float32, device=dev)
        csub = torch.empty(gsub.coeff_shape, dtype=torch.float32, device=dev)
        spl.forward(gsub, c_true, ysub, proj.basis)
        spl.adjoint(gsub, ysub, csub, proj.basis)
        a_ms = time_call(lambda: spl.forward(gsub, c_true, ysub, proj.basis))
        at_ms = time_call(lambda: spl.adjoint(gsub, ysub, csub, proj.basis))
        gsub.status()
        per_class[name] = {"views": cl["views"], "contributions_per_A": cl["pairs"], "A_ms": a_ms, "AT_ms": at_ms,
                           "A_gcontrib_s": cl["pairs"] / (a_ms * 1e-3) / 1e9,
                           "AT_gcontrib_s": cl["pairs"] / (at_ms * 1e-3) / 1e9}
        if name == "general":
            # the same A as the line integral of f itself (SPL_FP_DIRECT, the
            # exact alternative of the footprint form; not the headline)
            bd = spl.basis(n, spl.SPL_FP_DIRECT)
            spl.forward(gsub, c_true, ysub, bd)
            ad_ms = time_call(lambda: spl.forward(gsub, c_true, ysub, bd))
            gsub.status()
            per_class[name]["A_direct_ms"] = ad_ms
            per_class[name]["A_direct_gcontrib_s"] = cl["pairs"] / (ad_ms * 1e-3) / 1e9
            # the splat form (SPL_FP_TABLE: tabulated footprints, an
            # approximation) on the same views, and its distance to exact A
            bt = spl.basis(n, spl.SPL_FP_TABLE)
            yt = torch.empty_like(ysub)
            spl.forward(gsub, c_true, yt, bt)
            spl.adjoint(gsub, yt, csub, bt)
            at_t = time_call(lambda: spl.forward(gsub, c_true, yt, bt))
            att_t = time_call(lambda: spl.adjoint(gsub, yt, csub, bt))
            spl.forward(gsub, c_true, ysub, proj.basis)
            gsub.status()
            per_class[name]["A_table_ms"] = at_t
            per_class[name]["AT_table_ms"] = att_t
            per_class[name]["table_A_rel_l2_vs_exact"] = float((yt - ysub).norm() / ysub.norm())

    contrib_step = 2 * pairs  # A and A^T visit the same pairs
    value = replica_value(ws, contrib_step, ms)

    # end to end through the C ABI with host buffers: H2D of c and y from
    # pinned memory, A c and A^T y, D2H of both results, every step.  The
    # copies run on a copy stream: y's upload overlaps A, the download of
    # A c overlaps A^T; each step's uploads wait for the previous step's
    # downloads, which wait for its A and A^T (no buffer is overwritten
    # while in use).
    c_host = torch.tensor(wl.coeffs).pin_memory()
    y_host = y.cpu().pin_memory()
    out_y = torch.empty_like(y_host).pin_memory()
    out_c = torch.empty_like(c_host).pin_memory()
    c_dev = torch.empty_like(c_true)
    y_dev = torch.empty_like(y)
    e2e_steps = max(3, min(args.steps, 5))
    copy_s = torch.cuda.Stream()
    ev = {k: torch.cuda.Event() for k in ("c", "y", "a", "at")}
    torch.cuda.synchronize()
    e_start, e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    copy_s.wait_event(e_start)
    for _ in range(e2e_steps):
        with torch.cuda.stream(copy_s):
            c_dev.copy_(c_host, non_blocking=True)
            ev["c"].record(copy_s)
            y_dev.copy_(y_host, non_blocking=True)
            ev["y"].record(copy_s)
        stream.wait_event(ev["c"])
        proj.forward(c_dev, out=cg.q)
        ev["a"].record(stream)
        stream.wait_event(ev["y"])
        proj.adjoint(y_dev, out=cg.s)
        ev["at"].record(stream)
        with torch.cuda.stream(copy_s):
            copy_s.wait_event(ev["a"])
            out_y.copy_(cg.q, non_blocking=True)
            copy_s.wait_event(ev["at"])
            out_c.copy_(cg.s, non_blocking=True)
    stream.wait_stream(copy_s)
    e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e_start.elapsed_time(e_stop) / e2e_steps
    # the downloaded results against the same operators on device buffers
    ref_y, ref_c = torch.empty_like(y), torch.empty_like(c_true)
    proj.forward(c_true, out=ref_y)
    proj.adjoint(y, out=ref_c)
    torch.cuda.synchronize()
    e2e_diff = max(float((out_y.to(dev) - ref_y).norm() / ref_y.norm()),
                   float((out_c.to(dev) - ref_c).norm() / ref_c.norm()))
    h2d = c_host.numel() * 4 + y_host.numel() * 4
    d2h = out_y.numel() * 4 + out_c.numel() * 4

    clocks = sampler.summary()
    peaks = measured_peaks()
    max_mhz = (clocks.get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0)
    fp32_peak_tflops = SMS * FP32_LANES * 2 * max_mhz * 1e6 / 1e12
    # dominant kernel: the cell march of the general views (one launch per
    # A or A^T); its algorithmic FP32 work is the nodes it integrates plus
    # one FMA per contribution
    gen = classes.get("general", classes.get("separable"))
    flops_gen = (gen["pieces"] * NODES_PER_PIECE[n] * FLOP_PER_NODE[n]
                 + gen["flat_pieces"] * (n + 1) * FLOP_PER_FLAT_NODE[n] + gen["pairs"] * FLOP_PER_PAIR)
    pc_gen = per_class["general" if "general" in per_class else "separable"]
    if pc_gen["A_ms"] >= pc_gen["AT_ms"]:
        dominant, dom_ms = "k_forward_pviews (general views)", pc_gen["A_ms"]
    else:
        dominant = ("k_adjoint_bricks" if args.adjoint == "gather" else
                    "k_adjoint_pviews_scatter (general views)")
        dom_ms = pc_gen["AT_ms"]
    achieved = flops_gen / (dom_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                "traffic": NCU_TRAFFIC.get(dominant.split(" ")[0]),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz max SM clock" % max_mhz,
                "algorithmic_flop_per_launch": flops_gen,
                "launch_ms": dom_ms}
    n_sep = per_class.get("separable", {}).get("views", 0)
    n_gen = per_class.get("general", {}).get("views", 0)
    launches_step = ((2 if n_sep else 0) + (1 if n_gen else 0)      # A: z-resample + row gather, cell march
                     + (3 if n_sep else 0) + (1 if n_gen else 0)    # A^T: transpose + column gather + z-adjoint, scatter
                     + 2 * 2 + 2)                                   # two FP64 dots (2 kernels each), two CG updates

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "degree": n, "footprint": "exact quadrature",
                       "adjoint": args.adjoint,
                       "coeffs": list(wl.dims), "views": wl.geometry.n_views, "detector": [wl.geometry.nu,
                                                                                          wl.geometry.nv],
                       "contributions_per_A": pairs, "pieces_per_A": pieces, "flat_pieces_per_A": flat_pieces,
                       "l2": "256 MB buffer written between timed steps (outside the step events)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "s_per_recon_iter": ms / 1e3,
            "A_ms": fwd, "AT_ms": adj,
            "A_gcontrib_s": pairs / (fwd * 1e-3) / 1e9, "AT_gcontrib_s": pairs / (adj * 1e-3) / 1e9,
            "e2e": {"value": replica_value(ws, contrib_step, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "result_rel_diff": e2e_diff},
            "gpu_launches": args.steps * launches_step,
            "view_classes": per_class,
            "plane_build_s": plane_build_s,
            "clocks": clocks,
            "roofline": roofline,
            "wall_s_timed_region": t_wall}

    if args.mlp_steps > 0:
        line["mlp"] = mlp_measure(args, wl, geom, c_true, y, pairs, proj, dev)

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        wl.coeffs = wl.coeffs.astype(np.float64)
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_mlp_views(args):
    """The learned-footprint projector alone on a subset of the workload's
    views: one forward and one adjoint, timed with CUDA events."""
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import spl

    B.build()
    spl.lib()
    a, b = (int(v) for v in args.mlp_views.split(":"))
    wl = I.workload_tilt(args.degree)
    geom = spl.Geometry(wl.dims, wl.origin, wl.geometry.subset_views(np.arange(a, b)))
    c = torch.tensor(wl.coeffs, device="cuda")
    mlp = spl.Mlp(args.degree, max_batch=8192, seed=5)
    train_us = None
    if args.mlp_steps > 0:
        from paper_2511_11078_gb300 import learn

        data = learn.FootprintSet(args.degree, 1 << 22, seed=31, device=torch.device("cuda"))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        learn.train(mlp, data, steps=args.mlp_steps, batch=8192, lr0=3e-3, lr_min=1e-6)
        torch.cuda.synchronize()
        train_us = (time.perf_counter() - t0) / args.mlp_steps * 1e6
    bas = spl.basis(args.degree, spl.SPL_FP_MLP, mlp)
    y = torch.empty(geom.n_rays, device="cuda")
    cb = torch.empty(geom.coeff_shape, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    spl.forward(geom, c, y, bas)
    ev[1].record()
    spl.adjoint(geom, y, cb, bas)
    ev[2].record()
    torch.cuda.synchronize()
    geom.status()
    print(json.dumps({"mlp_views": [a, b], "A_ms": ev[0].elapsed_time(ev[1]), "AT_ms": ev[1].elapsed_time(ev[2]),
                      "pairs": spl.count_pairs(geom, args.degree), "train_steps": args.mlp_steps,
                      "train_us_per_step": train_us}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mlp_views:
        return run_mlp_views(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
