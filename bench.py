#!/usr/bin/env python3
"""Throughput of the local tone-mapping path on GB300 (one JSON line).

Default workload: one 4000 x 3000 (12 MP) float32 RGB synthetic WDR image,
64 bins, receptive-field half-sizes 8/32/128, plain forward. A step is one
whole forward (range, bins, integral image, integral histogram / fused sweep,
multi-field lookup, fusion, colour restoration) over one image.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank tone-maps its own
images: the path has no exchange step, so ranks are replicas (weak scaling).
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
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
sys.path.insert(0, ROOT)

METRIC = "megapixels/s at 12 MP (fwd; fwd+bwd; batched vs per-image) and % of HBM roofline"
WORKLOAD = dict(name="wdr-12mp-fwd", H=3000, W=4000, n_bins=64, radii=[8, 32, 128],
                decades=(-3.0, 5.0), seed=1)
# Algorithmic HBM bytes per pixel (float32 RGB): the path must read the input
# twice (the global range precedes binning) and write the output once.
PATH_BYTES_PER_PX = 36


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Replicas: every rank tone-maps its own images (the path has no exchange
# step); the job's time is the slowest rank's, its throughput all ranks' units
# over that time. These helpers are the whole multi-rank logic.
def dist_init(backend: str):
    """Join the process group when launched with WORLD_SIZE > 1."""
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return rank, world, local


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over the ranks (every rank gets it)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base: int, rank: int, j: int) -> int:
    """Seed of image j of `rank`: distinct images on every rank."""
    return base + rank * 2 + j


def job_rate(units_per_rank: float, world: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time (units/s / 1e6)."""
    return world * units_per_rank * steps / (ms_max / 1e3) / 1e6


# ------------------------------------------------------------ reference arm --
def oracle_rate(img, wl, budget_s: float, seed: int = 0, threads: int = 1):
    """Oracle MP/s on sampled pixels of the workload: the global pre-pass over
    the whole image plus direct per-pixel evaluation until `budget_s`, on
    `threads` host threads (the per-pixel loop; the pre-pass is serial)."""
    import oracle

    oracle.build()
    oracle.set_threads(threads)
    op = oracle.make_params(wl["n_bins"], wl["radii"], eps=float(np.float32(0.1)),
                            sat=float(np.float32(0.6)))
    H, W = img.shape[:2]
    rng = np.random.default_rng(seed)
    done, t0 = 0, time.perf_counter()
    chunk = 2048 * threads  # enough pixels per call that the serial pre-pass does not dominate
    # each call re-runs the O(N) pre-pass; its cost is part of the oracle
    while time.perf_counter() - t0 < budget_s:
        ys = rng.integers(0, H, chunk)
        xs = rng.integers(0, W, chunk)
        oracle.forward_pixels(img, op, xs, ys)
        done += chunk
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return done / dt / 1e6, done, dt


def oracle_c1_full(threads: int):
    """The oracle's whole forward over the 512 x 384 workload (32 bins, radii
    4/16/64) on `threads` host threads: (MP/s, seconds)."""
    import oracle
    import synth

    oracle.build()
    img = synth.wdr_image(384, 512, seed=0)
    op = oracle.make_params(32, [4, 16, 64], eps=float(np.float32(0.1)), sat=float(np.float32(0.6)))
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.forward(img, op)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return 384 * 512 / dt / 1e6, dt


def host_cores() -> int:
    return os.cpu_count() or 1


def cpu_baseline(img, wl, seconds: float) -> dict:
    """The oracle as it stands on this host: the 12 MP workload sampled on all
    cores and on one, and the 512 x 384 workload in full on all cores."""
    nproc = host_cores()
    r_all, n_all, dt_all = oracle_rate(img, wl, seconds * 0.45, threads=nproc)
    r_one, n_one, dt_one = oracle_rate(img, wl, seconds * 0.35, seed=1, threads=1)
    c1_rate, c1_s = oracle_c1_full(nproc)
    return {"value": r_all, "unit": "MP/s", "cores": nproc, "kind": "oracle",
            "sample": f"{n_all} pixels sampled uniformly from the 12 MP image, direct window loops "
                      f"over {nproc} threads, {dt_all:.1f} s (pre-pass serial)",
            "one_thread": {"value": r_one, "unit": "MP/s", "cores": 1,
                           "sample": f"{n_one} sampled pixels, {dt_one:.1f} s"},
            "c1_full": {"value": c1_rate, "unit": "MP/s", "cores": nproc, "seconds": c1_s,
                        "sample": "512 x 384, 32 bins, radii 4/16/64, whole forward"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth

    wl = WORKLOAD
    img = synth.wdr_image(wl["H"], wl["W"], seed=wl["seed"], decades=wl["decades"])
    budget = args.ref_seconds or max(2.0, min(20.0, 60.0 / max(args.steps + args.warmup, 1)))
    nproc = host_cores()
    for _ in range(args.warmup):
        oracle_rate(img, wl, budget / 4, threads=nproc)
    rates, pix, secs = [], 0, 0.0
    for k in range(args.steps):
        r, n, dt = oracle_rate(img, wl, budget, seed=k, threads=nproc)
        rates.append(r)
        pix += n
        secs += dt
    value = pix / secs / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "height": wl["H"], "width": wl["W"], "n_bins": wl["n_bins"],
                   "radii": wl["radii"], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "MP/s", "cores": nproc, "kind": "oracle",
                         "sample": f"{pix} pixels sampled uniformly from the 12 MP image, each "
                                   f"evaluated by direct window loops over {nproc} threads after the "
                                   "O(N) pre-pass"},
        "e2e": {"value": value, "unit": "MP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- ours --
def run_ours(args):
    import torch

    import paper_2102_01289_gb300 as tm
    import synth

    rank, world, local = dist_init("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tm.build()
    wl = WORKLOAD
    H, W = wl["H"], wl["W"]
    npx = H * W
    params = tm.make_params(wl["n_bins"], wl["radii"], eps=0.1, sat=0.6)
    ctx = tm.tm_create(params)
    tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, HIST_PATHS[args.hist_path])
    stream = torch.cuda.current_stream(dev)

    # two resident inputs > L2 each, alternated so no step reuses cached input
    imgs = [synth.wdr_image(H, W, seed=replica_seed(wl["seed"], rank, j), decades=wl["decades"]) for j in range(2)]
    xin = [torch.from_numpy(a).to(dev) for a in imgs]
    xout = [torch.empty_like(x) for x in xin]

    for i in range(args.warmup):
        tm.tm_forward(ctx, xin[i % 2], xout[i % 2], stream)
    torch.cuda.synchronize()
    launches_per_step = tm.tm_last_launch_count(ctx)

    # timed region: device time with CUDA events on the launching stream
    # (each forward replays the context's cached CUDA graph of its buffers)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist_barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        tm.tm_forward(ctx, xin[i % 2], xout[i % 2], stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    ms = e0.elapsed_time(e1)
    # per-stage device times: the same steps again, with the events the
    # library records on the launching stream after each stage (stage events
    # run the forward's launches one by one instead of its graph)
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 1)
    tm.tm_stage_times(ctx)  # reset
    for i in range(args.steps):
        tm.tm_forward(ctx, xin[i % 2], xout[i % 2], stream)
    torch.cuda.synchronize()
    stages = tm.tm_stage_times(ctx)
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 0)
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / args.steps
    value = job_rate(npx, world, args.steps, ms)

    # end to end through the public API with host buffers: page-locked host
    # in/out, the H2D copy of each step's input and the D2H of its result
    # inside every step. The stream of frames goes through
    # tm_forward_host_async (the next frame's upload and the previous frame's
    # download overlap each forward); the clock stops after the stream has
    # drained, so the pipeline's fill and drain are inside it.
    hin = [torch.from_numpy(a).pin_memory() for a in imgs]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    e2e_steps = max(args.steps, 30)
    for i in range(2):
        tm.tm_forward_host_async(ctx, hin[i].numpy(), hout[i].numpy(), stream)
    torch.cuda.synchronize()
    dist_barrier(world)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        tm.tm_forward_host_async(ctx, hin[i % 2].numpy(), hout[i % 2].numpy(), stream)
    stream.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = job_rate(npx, world, e2e_steps, e2e_s * 1e3)
    # the synchronous call, one frame at a time, for comparison
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        tm.tm_forward_host(ctx, hin[i % 2].numpy(), hout[i % 2].numpy(), stream)
    e2e_sync_s = max_over_ranks(time.perf_counter() - t0, world, dev)

    peak, peak_kind = load_peaks()
    # on the fused path the integral images run beside the sweep, in the SMs
    # its last segments leave idle: their stage time spans the sweep's tail and
    # is not a kernel of its own, so the dominant kernel is taken among the others
    own = {k: v for k, v in stages.items() if not (k == "integral_image" and "fused_sweep" in stages)}
    dominant = max(own.items(), key=lambda kv: kv[1])[0] if own else None
    dom_ms = stages.get(dominant, 0.0) / args.steps if dominant else 0.0
    # the roofline of the dominant kernel takes the path's algorithmic bytes per
    # pixel times the pixels one launch processes, over that kernel's mean time
    bpp = PATH_BYTES_PER_PX
    achieved = bpp * npx / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None
    traffic = load_traffic(dominant)
    # the dominant kernel is limited by instruction issue, not HBM: its warp
    # instructions per launch (ncu) over the SMs' issue slots in its time
    inst = load_profile(dominant, "warp_inst_per_launch")
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or None
    issue = None
    if inst and mhz and dom_ms > 0:
        slots = nsm * 4 * mhz * 1e6 * dom_ms / 1e3
        issue = {"warp_inst_per_launch": inst, "sms": nsm, "sm_mhz": mhz, "issue_slots": slots,
                 "frac": inst / slots, "warp_inst_per_px": inst / npx}
    line = {
        "metric": METRIC, "value": value, "unit": "MP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"], "height": H, "width": W, "channels": 3, "input": "float32",
                   "n_bins": wl["n_bins"], "radii": wl["radii"], "parallelism": "replicas",
                   "l2": "inputs larger than L2 (two 144 MB images alternated)",
                   "hist_path": "fused" if "fused_sweep" in stages else "materialised"},
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "bytes_per_px": bpp, "kernel_ms": dom_ms, "issue": issue},
        "path_roofline": {"bytes_per_px": PATH_BYTES_PER_PX,
                          "achieved": PATH_BYTES_PER_PX * npx / (ms_step / 1e3) / 1e9,
                          "peak": peak, "unit": "GB/s",
                          "frac": PATH_BYTES_PER_PX * npx / (ms_step / 1e3) / 1e9 / peak},
        "stages_ms_per_step": {k: v / args.steps for k, v in stages.items()},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "MP/s", "h2d_bytes_per_step": int(imgs[0].nbytes),
                "d2h_bytes_per_step": int(imgs[0].nbytes), "steps": e2e_steps,
                "api": "tm_forward_host_async (page-locked frames, stream drained inside the timing)",
                "synchronous_per_call": job_rate(npx, world, e2e_steps, e2e_sync_s * 1e3)},
        "gpu_launches": int(launches_per_step * args.steps),
    }
    tm.tm_destroy(ctx)
    if world == 1 and not args.no_legs:
        # the other legs of the metric, each against its per-image forward
        line["legs"] = {
            "fwd_bwd": leg_fwd_bwd(args, dev),
            "batch_video": leg_batch(args, dev, "batch-video"),
            "batch_uneven": leg_batch(args, dev, "batch-uneven"),
            "paper_preset": leg_paper_preset(args, dev),
        }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(imgs[0], wl, args.cpu_seconds)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- other workloads --
def _timed(fn, steps, stream):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _roof(bpp, npx, ms):
    peak, peak_kind = load_peaks()
    ach = bpp * npx / (ms / 1e3) / 1e9
    return {"bytes_per_px": bpp, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": peak_kind}


def leg_batch(args, dev, kind, steps=None, warmup=None):
    """Batched graph path vs per-image forward on the same images.
    batch-video: 120 1920x1080 FP16 frames (moving rectangles over a drifting
    ramp, per-frame noise), 32 bins, half-sizes 8/32/128, FP16 output.
    batch-uneven: 64 float32 images, W ~ U{640..4096}, 4:3 or 16:9, 64 bins.
    Inputs are rendered on the device (synth.wdr_device, the same recipe)."""
    import torch

    import paper_2102_01289_gb300 as tm
    import synth

    rank = dist_env()[0]
    steps = steps or max(3, min(args.steps, 5))
    warmup = warmup or 3
    tm.build()
    if kind == "batch-video":
        n = 120
        xs = [synth.wdr_device(1080, 1920, seed=7 + rank, device=dev, frame=f, dtype=torch.float16)
              for f in range(n)]
        params = tm.make_params(32, [8, 32, 128])
        name, bpp = "wdr-video-1080p-fp16-x120", 18
    else:
        sizes = synth.uneven_sizes(64, seed=rank)
        xs = [synth.wdr_device(h, w, seed=k + 100 * rank, device=dev) for k, (w, h) in enumerate(sizes)]
        params = tm.make_params(64, [8, 32, 128])
        name, bpp = "wdr-uneven-x64", 36
    npx = sum(x.shape[0] * x.shape[1] for x in xs)
    ys = [torch.empty_like(x) for x in xs]
    ctx = tm.tm_create(params)
    tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, HIST_PATHS[args.hist_path])
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(dev.index or 0)
    for _ in range(warmup):
        tm.tm_forward_batch(ctx, xs, ys, stream)
    launches = tm.tm_last_launch_count(ctx)
    # which batched pass(es) the images took: the fused sweep and/or the
    # materialised integral histogram (the per-size choice the library made)
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 1)
    tm.tm_stage_times(ctx)
    tm.tm_forward_batch(ctx, xs, ys, stream)
    passes = sorted({"batch": "fused", "batch_materialised": "materialised"}[k]
                    for k in tm.tm_stage_times(ctx) if k in ("batch", "batch_materialised"))
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 0)
    clocks.start()
    time.sleep(0.3)
    ms_batch = _timed(lambda i: tm.tm_forward_batch(ctx, xs, ys, stream), steps, stream)
    clk = clocks.stop()

    # per-image forward on the same images, after one untimed pass over all of
    # them (the first forward of each image size measures both histogram paths)
    def per_image(i):
        for x, y in zip(xs, ys):
            tm.tm_forward(ctx, x, y, stream)

    per_image(0)
    ms_single = _timed(per_image, max(1, steps // 2), stream)
    ms_reuse = None
    if kind == "batch-video":  # streaming variant: each frame binned over the previous frame's range
        tm.tm_set_option(ctx, tm.TM_OPT_REUSE_RANGE, 1)
        per_image(0)
        ms_reuse = _timed(per_image, max(1, steps // 2), stream)
        tm.tm_set_option(ctx, tm.TM_OPT_REUSE_RANGE, 0)
    tm.tm_destroy(ctx)
    del xs, ys
    rate = lambda ms: npx / (ms / 1e3) / 1e6  # noqa: E731
    return {
        "value": rate(ms_batch), "unit": "MP/s", "ms_per_step": ms_batch, "steps": steps, "warmup": warmup,
        "dtype": "f16" if kind == "batch-video" else "f32",
        "config": {"workload": name, "images": n if kind == "batch-video" else 64, "megapixels": npx / 1e6,
                   "n_bins": params.n_bins, "radii": [8, 32, 128], "path": "batched graph",
                   "histogram_passes": passes,
                   "l2": "inputs larger than L2", "inputs": "rendered on the device (synth.wdr_device)"},
        "per_image_forward": {"value": rate(ms_single), "unit": "MP/s", "ms": ms_single},
        "per_image_forward_reused_range": (
            {"value": rate(ms_reuse), "unit": "MP/s", "ms": ms_reuse} if ms_reuse else None),
        "batched_over_per_image": ms_single / ms_batch,
        "path_roofline": _roof(bpp, npx, ms_batch),
        "clocks": clk, "gpu_launches": int(launches * steps),
    }


def leg_fwd_bwd(args, dev, steps=None, warmup=None):
    """16 float32 1024x1024 images, 32 bins, half-sizes 8/32/128: one step is
    the batched forward (tm_forward_batch) plus the batched backward
    (tm_backward_batch: input and parameter gradients). Also timed: the same
    work as per-image calls, and the per-image forward alone."""
    import torch

    import paper_2102_01289_gb300 as tm
    import synth

    rank = dist_env()[0]
    steps = steps or max(3, min(args.steps, 10))
    warmup = warmup or 3
    tm.build()
    n, H, W = 16, 1024, 1024
    xs = [synth.wdr_device(H, W, seed=s + 16 * rank, device=dev) for s in range(n)]
    ys = [torch.empty_like(x) for x in xs]
    g = torch.Generator(device=dev)
    g.manual_seed(1234 + rank)
    gs = [torch.randn(x.shape, generator=g, device=dev) for x in xs]
    gins = [torch.empty_like(x) for x in xs]
    params = tm.make_params(32, [8, 32, 128])
    gp = torch.empty(3 + 2 * 3, device=dev)
    ctx = tm.tm_create(params)
    tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, HIST_PATHS[args.hist_path])
    # as in the autograd function: the backward of the images just forwarded
    # takes the forward's intermediates instead of recomputing them
    tm.tm_set_option(ctx, tm.TM_OPT_BACKWARD_REUSE, 1)
    stream = torch.cuda.current_stream(dev)

    def batched(i):
        tm.tm_forward_batch(ctx, xs, ys, stream)
        tm.tm_backward_batch(ctx, xs, gs, gins, gp, stream)

    def per_image(i):
        for x, y, gg, gi in zip(xs, ys, gs, gins):
            tm.tm_forward(ctx, x, y, stream)
            tm.tm_backward(ctx, x, gg, gi, gp, stream)

    def fwd(i):
        for x, y in zip(xs, ys):
            tm.tm_forward(ctx, x, y, stream)

    for _ in range(warmup):
        batched(0)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    ms_b = _timed(batched, steps, stream)
    clk = clocks.stop()
    ms_p = _timed(per_image, max(1, steps // 2), stream)
    ms_f = _timed(fwd, steps, stream)
    tm.tm_destroy(ctx)
    npx = n * H * W
    rate = lambda ms: npx / (ms / 1e3) / 1e6  # noqa: E731
    return {
        "value": rate(ms_b), "unit": "MP/s", "ms_per_step": ms_b, "steps": steps, "warmup": warmup,
        "dtype": "f32",
        "config": {"workload": "wdr-1mp-x16-fwd-bwd", "images": n, "height": H, "width": W,
                   "n_bins": 32, "radii": [8, 32, 128],
                   "path": "batched forward + batched backward (forward intermediates reused)",
                   "l2": "inputs larger than L2", "inputs": "rendered on the device (synth.wdr_device)"},
        "per_image_fwd_bwd": {"value": rate(ms_p), "unit": "MP/s", "ms": ms_p},
        "per_image_forward": {"value": rate(ms_f), "unit": "MP/s", "ms": ms_f},
        "path_roofline": _roof(36 + 48, npx, ms_b),
        "clocks": clk,
    }


def leg_paper_preset(args, dev, steps=None, warmup=None):
    """The paper's own setting at 12 MP: s = 5 fields halving from the whole
    image (rectangular), n = 5 bins, eps 0.1, sat 0.6 (tm_params_pyramid)."""
    import torch

    import paper_2102_01289_gb300 as tm
    import synth

    rank = dist_env()[0]
    steps = steps or max(3, min(args.steps, 10))
    warmup = warmup or 3
    tm.build()
    H, W = 3000, 4000
    xs = [synth.wdr_device(H, W, seed=3 + j + 2 * rank, device=dev, decades=(-3.0, 5.0)) for j in range(2)]
    ys = [torch.empty_like(x) for x in xs]
    params = tm.tm_params_pyramid(W, H, 5, 5)
    ctx = tm.tm_create(params)
    tm.tm_set_option(ctx, tm.TM_OPT_HIST_PATH, HIST_PATHS[args.hist_path])
    stream = torch.cuda.current_stream(dev)
    for i in range(warmup):
        tm.tm_forward(ctx, xs[i % 2], ys[i % 2], stream)
    launches = tm.tm_last_launch_count(ctx)
    tm.tm_set_option(ctx, tm.TM_OPT_STAGE_TIMING, 1)
    tm.tm_stage_times(ctx)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    ms = _timed(lambda i: tm.tm_forward(ctx, xs[i % 2], ys[i % 2], stream), steps, stream)
    clk = clocks.stop()
    stages = tm.tm_stage_times(ctx)
    tm.tm_destroy(ctx)
    npx = H * W
    return {
        "value": npx / (ms / 1e3) / 1e6, "unit": "MP/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "dtype": "f32",
        "config": {"workload": "wdr-12mp-paper-preset", "height": H, "width": W, "n_bins": 5,
                   "fields": [[int(params.rx[f]), int(params.ry[f])] for f in range(5)],
                   "hist_path": "materialised" if "integral_histogram" in stages else "fused",
                   "l2": "inputs larger than L2 (two 144 MB images alternated)",
                   "inputs": "rendered on the device (synth.wdr_device)"},
        "stages_ms_per_step": {k: v / steps for k, v in stages.items()},
        "path_roofline": _roof(PATH_BYTES_PER_PX, npx, ms),
        "clocks": clk, "gpu_launches": int(launches * steps),
    }


def run_leg(args, which):
    """One leg as its own JSON line (--workload)."""
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if which in ("batch-video", "batch-uneven"):
        d = leg_batch(args, dev, which, steps=args.steps, warmup=args.warmup)
    elif which == "fwd-bwd":
        d = leg_fwd_bwd(args, dev, steps=args.steps, warmup=args.warmup)
    else:
        d = leg_paper_preset(args, dev, steps=args.steps, warmup=args.warmup)
    line = {"metric": METRIC, "value": d.pop("value"), "unit": d.pop("unit"), "n_gpus": world,
            "steps": d.pop("steps"), "warmup": d.pop("warmup"), "ms_per_step": d.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": d.pop("dtype"),
            "data": "synthetic", "config": d.pop("config")}
    line.update(d)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def load_profile(kernel, key="bytes_per_launch"):
    """A per-launch figure of `kernel` from the committed ncu summary
    (profiles/traffic.json: DRAM bytes, warp instructions), or None once the
    kernel's source has changed since it was taken."""
    if not kernel:
        return None
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    return e.get(key)


def load_traffic(kernel):
    return load_profile(kernel, "bytes_per_launch")


HIST_PATHS = {"auto": 0, "fused": 1, "materialised": 2}


def kernel_source_hash(kernel):
    import hashlib

    import paper_2102_01289_gb300 as tm

    srcs = {"fused_sweep": "tm_sweep.cu", "lookup": "tm_lookup.cu", "bwd_pixel": "tm_backward.cu",
            "bwd_input": "tm_backward.cu", "fix_stats": "tm_integral.cu", "fix_write": "tm_integral.cu",
            "integral_histogram": "tm_integral.cu", "integral_image": "tm_integral.cu",
            "prep": "tm_prepass.cu", "range": "tm_prepass.cu"}
    f = os.path.join(tm.PKG, "csrc", srcs.get(kernel, ""))
    if not os.path.isfile(f):
        return None
    return hashlib.sha256(open(f, "rb").read()).hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the other legs of the metric (fwd+bwd, batches, paper preset)")
    ap.add_argument("--hist-path", choices=sorted(HIST_PATHS), default="auto",
                    help="histogram path: auto (the library measures both once), fused or materialised")
    ap.add_argument("--ref-seconds", type=float, default=0.0,
                    help="oracle sample per step of the reference arm (default: sized so the run takes ~1 min)")
    ap.add_argument("--workload", default="fwd-12mp",
                    choices=["fwd-12mp", "batch-video", "batch-uneven", "fwd-bwd", "paper-preset"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "fwd-12mp":
        return run_leg(args, args.workload)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
