#!/usr/bin/env python3
"""Benchmark of the B-spline x-ray transform (SplineSplat, arXiv 2511.11078).

Headline workload (one GPU): 512^3 FP32 cubic B-spline coefficients of a
12-ellipsoid phantom plus band-limited Gaussian noise texture; helical cone
beam, 720 views over 2 turns, helical pitch 0.5, 768x768 detector of pitch
0.8, source-to-centre 1000, source-to-detector 1500; data y = A c_true +
Gaussian noise (sigma = 1% of max).  One step = one CGLS iteration of the
least-squares problem of Eq. 5: one forward projection A, one matched
adjoint A^T, two FP64 inner products and the two CG vector updates, all on
the GPU with the exact quadrature footprint.  The inputs (c: 512 MB, y:
1.7 GB) are larger than L2, so no flush is needed between steps.

Metric: contributions (ray, basis pairs of Eq. 4) processed per second by
A and A^T, in G-contributions/s; also seconds per reconstruction iteration.

Besides the headline the line carries:
  * rel_l2_vs_oracle: the timed A and A^T against the FP64 oracle on a
    seeded, stratified sample of >= 4096 rays (A c_true on those rays; A^T
    of a y that is nonzero on them only);
  * cpu_baseline: that oracle work timed on the host cores;
  * roofline: the dominant kernel's algorithmic FP32 rate against the FP32
    peak measured in the same run by the library's FMA probe;
  * e2e: the same CGLS iteration with its state (x, r, p) resident in pinned
    host memory, uploaded before and downloaded after every step;
  * secondary: the 128^3 parallel tilt-series workload (244 views);
  * mlp: the learned footprint f_theta (Algorithm 1) trained in the run and
    used in A / A^T on the 256^3 circular cone-beam workload beside the
    quadrature footprint.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (as it stands) on the host cores,
each step a bounded sample of the same workload.  Under torchrun (N > 1)
the workload's views are split across the ranks, one GPU each (strong
scaling): A needs no exchange, A^T one all-reduce of the coefficients per
iteration and the FP64 inner products scalar all-reduces (NCCL); rank 0
prints the JSON line with the max-over-ranks step time and the whole job's
contributions.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import re
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
# views per batch of the scatter adjoint (FP32 atomics within a batch, FP64
# totals across batches when a geometry has more views than this)
ADJ_BATCH_VIEWS = 48


def launches_per_cg_step(n_views: int, scatter: bool = True) -> int:
    """Kernels of the library launched by one CGLS iteration on a cone
    geometry of n_views views: A (one launch), two FP64 dots (two kernels
    each), the x/r and p updates, and A^T: per batch of 48 views the scatter
    and the folds of its two layout copies, plus the batch's FP64 total
    (and the final rounding) when there is more than one batch; the brick
    gather is one launch."""
    if not scatter:
        return 1 + 4 + 2 + 1
    batched = n_views > ADJ_BATCH_VIEWS
    batches = -(-n_views // ADJ_BATCH_VIEWS) if batched else 1
    return 1 + 4 + 2 + batches * (3 + (1 if batched else 0)) + (1 if batched else 0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--adjoint", default="scatter", choices=["gather", "scatter"],
                    help="form of A^T: ray-driven scatter (float atomics, the library default) or brick gather")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle leg (cpu_baseline and rel_l2_vs_oracle)")
    ap.add_argument("--cpu-rays", type=int, default=4096, help="rays of the oracle sample (at least 4096 for the line)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 128^3 tilt-series block")
    ap.add_argument("--mlp-steps", type=int, default=200000,
                    help="Adam steps of the learned footprint trained before the MLP measurement (0: skip it)")
    ap.add_argument("--mlp-views", type=int, default=36,
                    help="views of the 256^3 cone workload (evenly spaced) the MLP projector is timed on")
    ap.add_argument("--mlp-recon-iters", type=int, default=10,
                    help="CGLS iterations of the learned-footprint vs quadrature reconstruction on those views "
                         "(0: skip it)")
    ap.add_argument("--profile-views", default=None, metavar="START:STOP[:STEP]",
                    help="only run A and A^T once each on views START..STOP-1 (every STEP-th) of the headline "
                         "workload (a small case for ncu) and print their times")
    ap.add_argument("--mlp-profile", default=None, metavar="START:STOP",
                    help="only run the learned-footprint projector (f_theta seeded 5, trained for --mlp-steps "
                         "steps first) once forward and once adjoint on views START..STOP-1 of the 256^3 cone "
                         "workload and print their times (a small case for profiling)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """The largest of the ranks' values (the step time of the slowest
    rank); the value itself at one rank."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(contributions_per_step: float, ms: float) -> float:
    """Whole-job throughput: the contributions all ranks together processed
    in one step, per second of the slowest rank's step time, in
    G-contributions/s."""
    return contributions_per_step / (ms * 1e-3) / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def csrc_sha16() -> str:
    """Hash of the CUDA sources and the C header: a kernel's ncu counters
    are reported only while the sources they were taken from are unchanged."""
    files = sorted(glob.glob(os.path.join(ROOT, "paper_2511_11078_gb300", "csrc", "*")))
    files.append(os.path.join(ROOT, "include", "spl.h"))
    h = hashlib.sha256()
    for fn in files:
        with open(fn, "rb") as f:
            h.update(os.path.basename(fn).encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu
    summary under profiles/ whose line
        traffic_bytes_per_launch <kernel> <workload> <bytes> csrc <sha16>
    names the current sources; None when there is none (or it is stale)."""
    sha = csrc_sha16()
    for fn in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(fn) as f:
            for line in f:
                m = re.match(r"\s*traffic_bytes_per_launch\s+(\S+)\s+(\S+)\s+([0-9.eE+]+)\s+csrc\s+([0-9a-f]+)",
                             line)
                if m and m.group(1) == kernel and m.group(2) == workload and m.group(4) == sha:
                    return float(m.group(3))
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
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            t = [x.strip() for x in ln.split(",")]
            if len(t) < 8:
                continue
            try:
                sm.append(float(t[0]))
                smax.append(float(t[1]))
                power.append(float(t[2]))
            except ValueError:
                continue
            for name, v in zip(names, t[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def gpu_index(local: int) -> int:
    if "CUDA_VISIBLE_DEVICES" in os.environ:
        try:
            return int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
        except (ValueError, IndexError):
            return local
    return local


# --------------------------------------------------------------------------
# the oracle side: geometry, stratified ray sample
# --------------------------------------------------------------------------
def oracle_geometry(oracle, geo):
    kw = dict(det_center=geo.det_center, det_u=geo.det_u, det_v=geo.det_v, nu=geo.nu, nv=geo.nv)
    if geo.kind == "parallel":
        return oracle.Geometry("parallel", direction=geo.src, **kw)
    return oracle.Geometry("cone", source=geo.src, **kw)


def stratified_rays(geo, count: int, seed: int) -> np.ndarray:
    """A seeded ray sample of a view geometry: 7/8 uniform over all rays, the
    rest on the detector's edge rows and columns, its centre, and the first
    and last views (ray ends, corner-truncated rays of cone views, the
    central ray)."""
    rng = np.random.default_rng(seed)
    n_rays = geo.n_rays
    nu, nv, nview = geo.nu, geo.nv, geo.n_views
    k_extra = count // 8
    uni = rng.choice(n_rays, count - k_extra, replace=False)
    views = rng.integers(0, nview, k_extra)
    views[: max(1, k_extra // 8)] = 0
    views[max(1, k_extra // 8): max(2, k_extra // 4)] = nview - 1
    which = rng.integers(0, 5, k_extra)
    iu = rng.integers(0, nu, k_extra)
    iv = rng.integers(0, nv, k_extra)
    iu = np.where(which == 0, 0, np.where(which == 1, nu - 1, iu))
    iv = np.where(which == 2, 0, np.where(which == 3, nv - 1, iv))
    iu = np.where(which == 4, nu // 2 + rng.integers(-2, 3, k_extra), iu)
    iv = np.where(which == 4, nv // 2 + rng.integers(-2, 3, k_extra), iv)
    extra = (views.astype(np.int64) * nv + iv) * nu + iu
    return np.unique(np.concatenate([uni, extra]).astype(np.int64))


def rel_l2(a, b) -> float:
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b)) / (nb if nb > 0 else 1.0)


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
    wl = I.workload_helical()
    coeffs = wl.coeffs.astype(np.float64)
    og = oracle_geometry(oracle, wl.geometry)
    # each step: oracle A on a ray sample plus A^T of a random y on it,
    # sized by a probe so the whole run takes a few minutes
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    probe = stratified_rays(wl.geometry, 128, seed=11)
    t0 = time.perf_counter()
    oracle.forward_subset(3, wl.dims, wl.origin, coeffs, og, probe, nthreads=threads)
    t_probe = 2.0 * (time.perf_counter() - t0)
    count = int(max(128, min(wl.geometry.n_rays, probe.size * per_step / max(t_probe, 1e-3))))
    rays = stratified_rays(wl.geometry, count, seed=12)
    ys = np.random.default_rng(13).uniform(0.0, 1.0, rays.size)

    def step():
        t = time.perf_counter()
        _, pairs = oracle.forward_subset(3, wl.dims, wl.origin, coeffs, og, rays, nthreads=threads)
        _, pairs_t = oracle.adjoint_subset(3, wl.dims, wl.origin, ys, og, rays, nthreads=threads)
        return time.perf_counter() - t, int(pairs.sum()) + int(pairs_t)

    for _ in range(args.warmup):
        step()
    tt, pp = 0.0, 0
    for _ in range(args.steps):
        t, p = step()
        tt += t
        pp += p
    value = pp / tt / 1e9
    sample = ("%d of %d rays (seeded stratified sample) per step: oracle A on them plus A^T of a random y on them"
              % (rays.size, wl.geometry.n_rays))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name + "-cubic", "degree": 3, "footprint": "exact quadrature (FP64)",
                       "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# FP32 peak: the library's FMA probe
# --------------------------------------------------------------------------
def fp32_peak(dev, local):
    import torch

    from paper_2511_11078_gb300 import spl

    out = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    sampler = ClockSampler(gpu_index(local))
    sampler.start()
    time.sleep(0.3)
    for packed in (False, True):
        spl.fp32_probe(out, packed, 4, 2048)  # warm-up
        best = 0.0
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flop = spl.fp32_probe(out, packed, 4, 1 << 18)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, flop / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        res["ffma2" if packed else "ffma"] = best
    sampler.stop()
    clk = sampler.summary()
    return {"tflops_ffma": res["ffma"], "tflops_ffma2": res["ffma2"], "peak": max(res.values()),
            "sms": spl.sm_count(), "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
            "probe": "spl_fp32_probe: 4 blocks/SM x 256 threads, 16 independent FMA chains per thread, 2^18 x 4 "
                     "iterations; best of 5 launches (CUDA events)"}


# --------------------------------------------------------------------------
# oracle leg: error of the timed operators and the CPU baseline
# --------------------------------------------------------------------------
def oracle_leg(args, wl, geom, ops, c_true, dev):
    """A c_true and A^T (y on a ray sample, zero elsewhere) by the timed GPU
    operators against the FP64 oracle on the same sample; the oracle's time
    is the CPU baseline."""
    import torch

    import oracle

    oracle.build()
    threads = os.cpu_count() or 1
    og = oracle_geometry(oracle, wl.geometry)
    rays = stratified_rays(wl.geometry, max(4096, args.cpu_rays), seed=2026)
    coeffs = c_true.cpu().numpy().astype(np.float64)
    ys = np.random.default_rng(2027).uniform(0.0, 1.0, rays.size).astype(np.float32)
    # GPU side (the operators as timed)
    yg = torch.empty(geom.n_rays, dtype=torch.float32, device=dev)
    ops.forward(c_true, yg)
    ymask = torch.zeros(geom.n_rays, dtype=torch.float32, device=dev)
    ymask[torch.tensor(rays, device=dev)] = torch.tensor(ys, device=dev)
    cg = torch.empty_like(c_true)
    ops.adjoint(ymask, cg)
    torch.cuda.synchronize()
    geom.status()
    ya = yg.cpu().numpy()[rays].astype(np.float64)
    ca = cg.cpu().numpy().astype(np.float64)
    del yg, ymask, cg
    # oracle side, timed
    t0 = time.perf_counter()
    yref, pairs = oracle.forward_subset(3, wl.dims, wl.origin, coeffs, og, rays, nthreads=threads)
    t1 = time.perf_counter()
    cref, pairs_t = oracle.adjoint_subset(3, wl.dims, wl.origin, ys.astype(np.float64), og, rays,
                                          nthreads=threads)
    t2 = time.perf_counter()
    total = int(pairs.sum()) + int(pairs_t)
    err = {"A": rel_l2(ya, yref), "AT": rel_l2(ca.reshape(-1), cref.reshape(-1)),
           "rays": int(rays.size), "pairs": int(pairs.sum()),
           "sample": "%d rays of the %s workload, seeded and stratified (7/8 uniform; detector edge rows and "
                     "columns, centre, first and last views): A c_true on them, and A^T of a uniform(0,1) y on "
                     "them (zero elsewhere)" % (rays.size, wl.name)}
    cpu = {"value": total / (t2 - t0) / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": "the %d-ray sample of rel_l2_vs_oracle: oracle A on it (%.1f s) plus A^T of y on it (%.1f s), "
                     "%d pairs in all" % (rays.size, t1 - t0, t2 - t1, total)}
    return err, cpu


# --------------------------------------------------------------------------
# end to end: the CGLS iteration with host-resident state
# --------------------------------------------------------------------------
def e2e_leg(cg, steps, stream):
    """Each step uploads the CGLS state (x, r, p) from pinned host memory,
    runs the iteration through the library's entry points, and downloads the
    updated x, r and p (and the FP64 scalar gamma).  p is needed by A at the
    start and rewritten at the end, so its copies stand in the step; x and r
    are first used after A (the x/r update) and final after it, so their
    upload runs on a copy stream beside A and their download beside A^T."""
    import torch

    hx, hr, hp = (t.cpu().pin_memory() for t in (cg.x, cg.r, cg.p))
    hg = torch.zeros(1, dtype=torch.float64).pin_memory()
    copy = torch.cuda.Stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        # x, r: the previous step is done with them (A^T read r)
        copy.wait_stream(stream)
        with torch.cuda.stream(copy):
            cg.x.copy_(hx, non_blocking=True)
            cg.r.copy_(hr, non_blocking=True)
        up = torch.cuda.Event()
        up.record(copy)
        cg.p.copy_(hp, non_blocking=True)

        def mark(i):
            if i == 1:  # after A, before the x/r update
                stream.wait_event(up)
            elif i == 2:  # x and r final for this step
                done = torch.cuda.Event()
                done.record(stream)
                copy.wait_event(done)
                with torch.cuda.stream(copy):
                    hx.copy_(cg.x, non_blocking=True)
                    hr.copy_(cg.r, non_blocking=True)

        cg.step(mark)
        hp.copy_(cg.p, non_blocking=True)
        hg.copy_(cg.gamma, non_blocking=True)
    stream.wait_stream(copy)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    nb = (hx.numel() + hr.numel() + hp.numel()) * 4
    return ms, nb, nb + 8, bool(np.isfinite(hg.numpy()).all())


# --------------------------------------------------------------------------
# secondary workload: the 128^3 tilt series
# --------------------------------------------------------------------------
def secondary_tilt(dev):
    import torch

    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import spl
    from paper_2511_11078_gb300.recon import CGLS, Projector

    n = 3
    wl = I.workload_tilt(n)
    geom = spl.Geometry(wl.dims, wl.origin, wl.geometry)
    proj = Projector(geom, n)
    c_true = torch.tensor(wl.coeffs, device=dev)
    t0 = time.perf_counter()
    spl.prepare(geom, proj.basis)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    y = proj.forward(c_true)
    pairs, pieces, flat_pieces = spl.count_work(geom, n)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def time_call(fn, reps=5):
        out = []
        for _ in range(reps):
            flush.fill_(1.0)
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            fn()
            t1.record(stream)
            torch.cuda.synchronize()
            out.append(t0.elapsed_time(t1))
        return statistics.median(out)

    cg = CGLS(proj, y)
    for _ in range(3):
        cg.step()
    step_ms = time_call(cg.step)
    a_ms = time_call(lambda: proj.forward(c_true, out=cg.q))
    at_ms = time_call(lambda: proj.adjoint(y, out=cg.s))
    geom.status()
    src = np.asarray(wl.geometry.src)
    flat = np.any(src == 0.0, axis=1)
    classes = {}
    for name, views in (("separable", np.nonzero(flat)[0]), ("general", np.nonzero(~flat)[0])):
        gsub = spl.Geometry(wl.dims, wl.origin, wl.geometry.subset_views(views))
        p_, _, _ = spl.count_work(gsub, n)
        ysub = torch.empty(gsub.n_rays, dtype=torch.float32, device=dev)
        csub = torch.empty(gsub.coeff_shape, dtype=torch.float32, device=dev)
        spl.forward(gsub, c_true, ysub, proj.basis)
        spl.adjoint(gsub, ysub, csub, proj.basis)
        am = time_call(lambda: spl.forward(gsub, c_true, ysub, proj.basis))
        atm = time_call(lambda: spl.adjoint(gsub, ysub, csub, proj.basis))
        rec = {"views": int(len(views)), "contributions_per_A": p_, "A_ms": am, "AT_ms": atm,
               "A_gcontrib_s": p_ / am / 1e6, "AT_gcontrib_s": p_ / atm / 1e6}
        if name == "general":
            bd = spl.basis(n, spl.SPL_FP_DIRECT)
            spl.forward(gsub, c_true, ysub, bd)
            rec["A_direct_ms"] = time_call(lambda: spl.forward(gsub, c_true, ysub, bd))
        gsub.status()
        classes[name] = rec
    return {"workload": "tilt-128^3-cubic-parallel-244x192^2", "contributions_per_A": pairs,
            "cg_step_ms": step_ms, "gcontrib_s": 2 * pairs / step_ms / 1e6,
            "A_ms": a_ms, "AT_ms": at_ms, "A_gcontrib_s": pairs / a_ms / 1e6, "AT_gcontrib_s": pairs / at_ms / 1e6,
            "plane_build_s": build_s, "view_classes": classes,
            "l2": "256 MB buffer written before each timed call (outside its events)"}


# --------------------------------------------------------------------------
# learned footprint: train f_theta (Algorithm 1), then use it in A / A^T on
# the 256^3 circular cone-beam workload beside the quadrature footprint
# --------------------------------------------------------------------------
def mlp_block(args, dev, with_oracle: bool):
    import torch

    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import learn, spl
    from paper_2511_11078_gb300.recon import Projector

    n = 3
    t0 = time.perf_counter()
    val = learn.FootprintSet(n, 1 << 18, seed=32, device=dev)
    mlp = spl.Mlp(n, max_batch=8192, seed=5)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    data = learn.train_recipe(mlp, n, scale=args.mlp_steps / learn.RECIPE["steps"], device=dev)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    mlp.status()
    acc = learn.evaluate(mlp, val)
    recon = None
    if args.mlp_recon_iters > 0:
        from paper_2511_11078_gb300 import experiment

        rviews = np.linspace(0, 360, args.mlp_views, endpoint=False).astype(int)
        recon = experiment.mlp_vs_quadrature(mlp, iters=args.mlp_recon_iters, views=rviews, device=dev)
    wl = I.workload_cone()
    views = np.linspace(0, wl.geometry.n_views, args.mlp_views, endpoint=False).astype(int)
    geo = wl.geometry.subset_views(views)
    geom = spl.Geometry(wl.dims, wl.origin, geo)
    pq = Projector(geom, n)
    pm = Projector(geom, n, spl.SPL_FP_MLP, mlp)
    c = torch.tensor(wl.coeffs, device=dev)
    pairs = spl.count_pairs(geom, n)
    yq, ym = torch.empty(geom.n_rays, device=dev), torch.empty(geom.n_rays, device=dev)
    cq, cm = torch.empty_like(c), torch.empty_like(c)
    pq.forward(c, out=yq)
    pm.forward(c, out=ym)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    q_a = timed(lambda: pq.forward(c, out=yq))
    q_at = timed(lambda: pq.adjoint(yq, out=cq))
    m_a = timed(lambda: pm.forward(c, out=ym))
    m_at = timed(lambda: pm.adjoint(yq, out=cm))
    geom.status()
    out = {"footprint": "f_theta 5-64-64-64-1 SiLU, BF16 weights/activations, FP32 accumulation (tcgen05, "
                        "accumulator in TMEM)", "dataset_s": t1 - t0,
           "workload": "%s-cubic, %d of %d views (evenly spaced)" % (wl.name, len(views), wl.geometry.n_views),
           "contributions_per_A": pairs,
           "quad": {"A_ms": q_a, "AT_ms": q_at, "A_gcontrib_s": pairs / q_a / 1e6, "AT_gcontrib_s": pairs / q_at / 1e6},
           "mlp": {"A_ms": m_a, "AT_ms": m_at, "A_gcontrib_s": pairs / m_a / 1e6, "AT_gcontrib_s": pairs / m_at / 1e6,
                   "tensor_tflops_A": pairs * MLP_FLOP_PER_PAIR / m_a / 1e9},
           "s_per_recon_iter_full_360_views": {"quad": (q_a + q_at) / 1e3 * wl.geometry.n_views / len(views),
                                               "mlp": (m_a + m_at) / 1e3 * wl.geometry.n_views / len(views)},
           "train": "Algorithm 1, support-masked, importance-sampled, two rounds of hard-example mining "
                    "(learn.RECIPE; step counts x %.3g)" % (args.mlp_steps / learn.RECIPE["steps"]),
           "train_steps": args.mlp_steps, "train_batch": 8192, "train_samples_final": data.count, "train_s": t2 - t1,
           "footprint_held_out": "%d samples of Algorithm 1's distribution, errors where the exact footprint is "
                                 "evaluated (masked by the exact support, as in the projector)" % val.count,
           "footprint_max_abs_over_peak": acc["max_abs_rel_peak"], "footprint_rms": acc["rms"],
           "A_rel_l2_vs_exact": float((ym - yq).norm() / yq.norm()),
           "AT_rel_l2_vs_exact": float((cm - cq).norm() / cq.norm())}
    if recon is not None:
        out["recon_psnr"] = recon
    if with_oracle:
        import oracle

        og = oracle_geometry(oracle, geo)
        rays = stratified_rays(geo, 1024, seed=2030)
        yref, _ = oracle.forward_subset(n, wl.dims, wl.origin, wl.coeffs.astype(np.float64), og, rays,
                                        nthreads=os.cpu_count() or 1)
        out["A_rel_l2_vs_oracle"] = {"mlp": rel_l2(ym.cpu().numpy()[rays], yref),
                                     "quad": rel_l2(yq.cpu().numpy()[rays], yref), "rays": int(rays.size)}
    return out


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
    from paper_2511_11078_gb300 import shard, spl

    B.build()
    spl.lib()
    n = 3
    t0 = time.perf_counter()
    wl = I.workload_helical()
    workload_s = time.perf_counter() - t0
    form = spl.SPL_ADJ_GATHER if args.adjoint == "gather" else spl.SPL_ADJ_SCATTER
    # the views of the workload split across the ranks (all of them at one
    # rank): A on a rank's views needs no exchange, A^T one sum over ranks
    ops = shard.ShardedProjector(wl.dims, wl.origin, wl.geometry, rank, ws, n, spl.basis(n, adjoint=form))
    geom = ops.geom
    c_true = torch.tensor(wl.coeffs, device=dev)
    y_clean = torch.empty(geom.n_rays, dtype=torch.float32, device=dev)
    ops.forward(c_true, y_clean)
    ymax = torch.tensor([float(y_clean.max())], dtype=torch.float64, device=dev)
    if ws > 1:
        torch.distributed.all_reduce(ymax, op=torch.distributed.ReduceOp.MAX)
    gen = torch.Generator(device=dev)
    gen.manual_seed(I.SEED_BASE + 5 + 1000 * rank)
    sigma = 0.01 * float(ymax.item())
    y = y_clean + sigma * torch.randn(y_clean.shape, generator=gen, device=dev)
    del y_clean
    work = torch.tensor(spl.count_work(geom, n), dtype=torch.float64, device=dev)
    geom.status()
    if ws > 1:
        torch.distributed.all_reduce(work)
    pairs, pieces, flat_pieces = (int(v) for v in work.tolist())

    cg = shard.ShardedCGLS(ops, y, c_true.shape)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        cg.step()
    torch.cuda.synchronize()
    geom.status()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_index(local))
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        cg.step(lambda i, k=k: ev[k][i].record(stream))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if ws > 1:
        torch.distributed.barrier()
    sampler.stop()
    geom.status()
    step_ms = [ev[k][0].elapsed_time(ev[k][4]) for k in range(args.steps)]
    fwd = statistics.median([ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)])
    adj = statistics.median([ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps)])
    ms = max_over_ranks(sum(step_ms) / args.steps, ws, dev)
    contrib_step = 2 * pairs  # A and A^T visit the same pairs (all ranks together)
    value = job_value(contrib_step, ms)
    clocks = sampler.summary()

    # end to end: the same iteration with host-resident state
    e2e_steps = max(1, min(args.steps, 2))
    e2e_ms, h2d, d2h, e2e_ok = e2e_leg(cg, e2e_steps, stream)
    e2e_ms = max_over_ranks(e2e_ms, ws, dev)
    geom.status()

    peak = fp32_peak(dev, local)
    # dominant kernel: the slower of A (k_forward_views) and A^T
    # (k_adjoint_views_scatter) on the cone views; its algorithmic FP32 work
    # is the nodes it integrates plus one FMA per contribution (this rank's
    # share of the work: the launch covers its views)
    flops = (pieces * NODES_PER_PIECE[n] * FLOP_PER_NODE[n] + flat_pieces * (n + 1) * FLOP_PER_FLAT_NODE[n]
             + pairs * FLOP_PER_PAIR) / ws
    if fwd >= adj:
        kname, dom_ms = "k_forward_views", fwd
    else:
        kname, dom_ms = ("k_adjoint_bricks" if args.adjoint == "gather" else "k_adjoint_views_scatter"), adj
    achieved = flops / (dom_ms * 1e-3) / 1e12
    workload_tag = wl.name + "-cubic"
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak["peak"], "unit": "TFLOP/s",
                "frac": achieved / peak["peak"], "traffic": ncu_traffic(kname, workload_tag),
                "peak_source": "measured in this run by the library's FP32 FMA probe (%d SMs; scalar FFMA %.1f, "
                               "packed FFMA2 %.1f TFLOP/s; the larger is the peak)"
                               % (peak["sms"], peak["tflops_ffma"], peak["tflops_ffma2"]),
                "algorithmic_flop_per_launch": flops, "launch_ms": dom_ms, "csrc_sha16": csrc_sha16()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_tag, "degree": n, "footprint": "exact quadrature",
                       "adjoint": args.adjoint, "coeffs": list(wl.dims), "views": wl.geometry.n_views,
                       "detector": [wl.geometry.nu, wl.geometry.nv], "geometry": "helical cone, 2 turns, pitch 0.5, "
                       "SOD 1000, SDD 1500, detector pitch 0.8",
                       "contributions_per_A": pairs, "pieces_per_A": pieces, "flat_pieces_per_A": flat_pieces,
                       "l2": "inputs larger than L2 (c 512 MB, y 1.7 GB); no flush",
                       "parallelism": ("views sharded over %d GPUs (A: no exchange; A^T: one all-reduce of c; "
                                       "FP64 dots: scalar all-reduces)" % ws) if ws > 1 else "single GPU"},
            "s_per_recon_iter": ms / 1e3,
            "A_ms": fwd, "AT_ms": adj,
            "A_gcontrib_s": pairs / (fwd * 1e-3) / 1e9, "AT_gcontrib_s": pairs / (adj * 1e-3) / 1e9,
            "e2e": {"value": job_value(contrib_step, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": e2e_steps,
                    "what": "the CGLS iteration with x, r, p in pinned host memory, uploaded and downloaded "
                            "(with gamma) in every step: p before A and after the p update, x and r on a copy "
                            "stream beside A (upload) and beside A^T (download)", "finite": e2e_ok},
            "gpu_launches": args.steps * launches_per_cg_step(ops.v1 - ops.v0, args.adjoint == "scatter"),
            "clocks": clocks,
            "roofline": roofline,
            "fp32_probe": peak,
            "workload_s": workload_s,
            "wall_s_timed_region": t_wall}
    del cg
    torch.cuda.empty_cache()

    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        err, cpu = oracle_leg(args, wl, geom, ops, c_true, dev)
        line["rel_l2_vs_oracle"] = err
        line["cpu_baseline"] = cpu
    del c_true, y, geom, ops
    torch.cuda.empty_cache()
    if not args.no_secondary:
        line["secondary"] = secondary_tilt(dev)
    if args.mlp_steps > 0:
        line["mlp"] = mlp_block(args, dev, with_oracle=(rank == 0 and not args.no_cpu_baseline and ws == 1))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_profile_views(args):
    """A and A^T once each on a subset of the headline workload's views (the
    full volume and detector): a small case for ncu."""
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import spl

    B.build()
    spl.lib()
    parts = [int(v) for v in args.profile_views.split(":")]
    a, b = parts[0], parts[1]
    step = parts[2] if len(parts) > 2 else 1
    wl = I.workload_helical()
    geom = spl.Geometry(wl.dims, wl.origin, wl.geometry.subset_views(np.arange(a, b, step)))
    bas = spl.basis(3, adjoint=spl.SPL_ADJ_GATHER if args.adjoint == "gather" else spl.SPL_ADJ_SCATTER)
    c = torch.tensor(wl.coeffs, device="cuda")
    y = torch.empty(geom.n_rays, device="cuda")
    cb = torch.empty(geom.coeff_shape, device="cuda")
    pairs, pieces, _ = spl.count_work(geom, 3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    spl.forward(geom, c, y, bas)
    ev[1].record()
    spl.adjoint(geom, y, cb, bas)
    ev[2].record()
    torch.cuda.synchronize()
    geom.status()
    a_ms, at_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    print(json.dumps({"profile_views": [a, b, step], "workload": wl.name + "-cubic", "A_ms": a_ms, "AT_ms": at_ms,
                      "pairs": pairs, "pieces": pieces, "A_gcontrib_s": pairs / a_ms / 1e6,
                      "AT_gcontrib_s": pairs / at_ms / 1e6, "csrc_sha16": csrc_sha16()}), flush=True)
    return 0


def run_mlp_profile(args):
    """The learned-footprint projector alone on a subset of the 256^3 cone
    workload's views: one forward and one adjoint, timed with CUDA events."""
    import torch

    from paper_2511_11078_gb300 import build as B
    from paper_2511_11078_gb300 import inputs as I
    from paper_2511_11078_gb300 import learn, spl

    B.build()
    spl.lib()
    a, b = (int(v) for v in args.mlp_profile.split(":"))
    wl = I.workload_cone()
    geom = spl.Geometry(wl.dims, wl.origin, wl.geometry.subset_views(np.arange(a, b)))
    c = torch.tensor(wl.coeffs, device="cuda")
    mlp = spl.Mlp(3, max_batch=8192, seed=5)
    if args.mlp_steps > 0:
        data = learn.FootprintSet(3, 1 << 22, seed=31, device=torch.device("cuda"))
        learn.train(mlp, data, steps=args.mlp_steps, batch=8192, lr0=3e-3, lr_min=1e-6)
    bas = spl.basis(3, spl.SPL_FP_MLP, mlp)
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
    print(json.dumps({"mlp_profile": [a, b], "A_ms": ev[0].elapsed_time(ev[1]), "AT_ms": ev[1].elapsed_time(ev[2]),
                      "pairs": spl.count_pairs(geom, 3), "train_steps": args.mlp_steps}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_views:
        return run_profile_views(args)
    if args.mlp_profile:
        return run_mlp_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
