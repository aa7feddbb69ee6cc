"""Benchmark of the resampling hot path on GB300.

One step = the batched, autotuned, reduced-precision form: 256 RGB uint8
images, H and W uniform on 64..2048, one scale per image uniform on [0.5, 4),
methods alternating bilinear / bicubic, resampled by the library's
replayable batch plan (one persistent launch per class, recorded as one CUDA
graph) with item shapes chosen by rs_autotune_batched before the timed
region. value = output pixels per step (an RGB pixel counts once) / device
time of the step, in Gpixels/s, whole job over all ranks. L2 is flushed (a
256 MB write) before every timed step, outside the step's events; a step's
inputs and outputs (6.6 GB) are far larger than L2 anyway.

Beside it (same run, "extras"): the paper's plain one-thread-per-pixel kernel
on FP32 copies of the same 256 images (the same accuracy: max / mean error
against the FP64 oracle reported for both), the same batch as one launch per
image, the RGB uint8 4096x4096 step (bicubic x2, bicubic x1.7, nearest x2)
with its dominant kernel's roofline, the single-channel 8192x8192 field in
FP32 / FP16 / BF16, the 512x512 uint8 bilinear x2 latency (direct and CUDA
graph replay), NCHW FP32 forward / backward / antialiased downscale.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
batch (bands of output rows of 16 of its images) on this host's cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "output Gpixels/s and % of HBM roofline, batched/low-precision vs plain FP32, at stated error"
BATCH_WORKLOAD = ("batch256_rgb_u8: 256 RGB uint8 images, H, W ~ U{64..2048}, scale ~ U[0.5, 4), "
                  "bilinear / bicubic alternating, smooth-field pixels (seed 4)")
RGB_OPS = (("bicubic_x2", "bicubic", 2.0), ("bicubic_x1.7", "bicubic", 1.7), ("nearest_x2", "nearest", 2.0))
FALLBACK_HBM_GBS = 6800.0
KERNEL_NAMES = {"window": "k_win", "stream": "k_stream", "tiled": "k_tiled", "gather": "k_nearest",
                "plain": "k_plain"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the batch plan with the default item shape")
    ap.add_argument("--tile-sweep", action="store_true",
                    help="the paper's tiling experiment on this GPU: an 800x800 uint8 image, bilinear at scales "
                         "2..10, the paper's kernel (one thread per output pixel) over block shapes, against "
                         "AUTO; prints a markdown table and exits")
    ap.add_argument("--ops-only", nargs="?", const="batch", default=None,
                    choices=["batch", "rgb", "nchw", "backward", "float", "sweep", "serving"],
                    help="profiling driver: run warmup + steps untimed launches of the 256-image batch plan "
                         "(batch, the default), of the three RGB 4096 resizes (rgb), of the NCHW FP32 forward "
                         "or backward x2 / x0.5 (nchw, backward), of the float 8192 bicubic x2 in FP32 / "
                         "FP16 / BF16 (float), of the paper's kernel with 32x4 and 4x32 blocks on the "
                         "800x800 uint8 bilinear x4 of the tiling study (sweep) or of the antialiased serving "
                         "downscales of 16 1920x1080 uint8 frames (serving: bicubic to 398x224 uint8, bilinear "
                         "to 455x256 normalised FP16), and exit")
    ap.add_argument("--flush-between", action="store_true",
                    help="profiling drivers only: write a 256 MB buffer after every launch, so that the next "
                         "launch's DRAM writes show the L2 write-back of the previous launch's output")
    ap.add_argument("--batch-images", type=int, default=256,
                    help="profiling drivers only: the first N images of the batch (a smaller capture)")
    return ap.parse_args()


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# --------------------------------------------------------------------------
# Distributed plumbing (one process per GPU; replicas, no data-path collective)

def dist_init(n):
    import torch
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(units_per_step: int, steps: int, local_seconds: float, world: int) -> tuple[float, float]:
    """Whole-job throughput: every rank processes units_per_step units per
    step; the job time is the slowest rank's time. Returns (units per
    second over all ranks, job seconds)."""
    job_s = max_over_ranks(local_seconds, world)
    return units_per_step * steps * world / job_s, job_s


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# Clock sampling during the timed region

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = open(os.devnull if False else "/tmp/rs_clocks_%d.csv" % os.getpid(), "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.out.name):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# GPU arm

# Source files each profiled kernel is built from (a change to any of them
# voids its recorded DRAM traffic).
KERNEL_SOURCES = {
    "k_batched_window": ["batched.cu", "win_body.cuh", "tile_body.cuh", "aa_wide.cuh", "rs_common.cuh", "rs_internal.h"],
    "k_win": ["win.cu", "win_body.cuh", "rs_common.cuh", "rs_internal.h"],
    "k_stream": ["stream.cu", "rs_common.cuh", "rs_internal.h"],
    "k_tiled": ["tiled.cu", "tile_body.cuh", "rs_common.cuh", "rs_internal.h"],
    "k_nearest": ["nearest.cu", "rs_common.cuh", "rs_internal.h"],
}


def kernel_source_sha(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = ROOT / "paper_1001_1718_gb300" / "csrc"
    for name in KERNEL_SOURCES.get(kernel, sorted(p.name for p in csrc.glob("*"))):
        h.update((csrc / name).read_bytes())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    p = ROOT / "profiles" / f"traffic_{kernel}_{workload}.txt"
    if not p.exists():
        return None
    kv = {}
    for line in p.read_text().splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha") != kernel_source_sha(kernel):
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def out_hw(n, s):
    return max(1, int(math.floor(n * s)))


class Flusher:
    def __init__(self, torch, dev):
        self.buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def __call__(self):
        self.buf.fill_(1)


def time_ops(torch, stream, ops, steps, warmup, flush):
    """ops: list of (name, fn). Each timed step flushes L2, then runs every op
    between its own pair of events. Returns per-op lists of ms."""
    for _ in range(warmup):
        for _, fn in ops:
            fn()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in ops]
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for s in range(steps):
            flush()
            for k, (_, fn) in enumerate(ops):
                ev[s][k][0].record(stream)
                fn()
                ev[s][k][1].record(stream)
    torch.cuda.synchronize()
    return {name: [ev[s][k][0].elapsed_time(ev[s][k][1]) for s in range(steps)]
            for k, (name, _) in enumerate(ops)}


def torch_index(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.int64)).cuda()


class Batch:
    """The 256-image ragged batch: host pixels, device inputs and outputs."""

    def __init__(self, torch, workloads, dev, n=256):
        self.items = workloads.batch_spec(seed=4)[:n]
        self.imgs = workloads.batch_images(self.items)
        self.srcs = [torch.from_numpy(im).to(dev) for im in self.imgs]
        self.outs = [torch.empty((it.Ho, it.Wo, 3), dtype=torch.uint8, device=dev) for it in self.items]
        self.methods = [workloads.METHOD_NAMES[it.method] for it in self.items]
        self.in_bytes = sum(x.numel() for x in self.srcs)
        self.out_bytes = sum(y.numel() for y in self.outs)
        self.out_px = sum(it.Ho * it.Wo for it in self.items)


def batch_errors(oracle, batch, outs, dtype="u8", n=512, every=16):
    """max / mean |gpu - FP64 oracle| (and uint8 steps off the rounded
    oracle) on n sampled points of every `every`-th image."""
    from paper_1001_1718_gb300 import workloads
    err, steps, tot, cnt = 0.0, 0.0, 0.0, 0
    for k in range(0, len(batch.items), every):
        it = batch.items[k]
        ys, xs = workloads.sample_points(k, it.Ho, it.Wo, n)
        ref = oracle.resize_points(batch.imgs[k].astype(np.float64), it.Ho, it.Wo, it.method, 0, -0.5, ys, xs)
        got = outs[k][torch_index(ys), torch_index(xs)].double().cpu().numpy()
        d = np.abs(got - ref)
        err, tot, cnt = max(err, float(d.max())), tot + float(d.sum()), cnt + d.size
        if dtype == "u8":
            steps = max(steps, float(np.abs(got - oracle.quantize_u8(ref)).max()))
    r = {"max_abs_vs_f64": err, "mean_abs_vs_f64": tot / max(1, cnt),
         "points": cnt, "images": len(range(0, len(batch.items), every))}
    if dtype == "u8":
        r["max_steps_vs_rounded_oracle"] = steps
    return r


def profile_ops(args, torch, rs, workloads, dev):
    """Untimed launches for profiling under ncu."""
    if args.ops_only == "nchw":
        xn = torch.from_numpy(workloads.workload_nchw_512(seed=5).astype(np.float32)).to(dev)
        ops = []
        for method in ("bilinear", "bicubic"):
            for s in (2.0, 0.5):
                Ho = int(512 * s)
                y = torch.empty((32, 3, Ho, Ho), dtype=torch.float32, device=dev)
                ops.append(lambda y=y, m=method, Ho=Ho: rs.resize(xn, (Ho, Ho), m, layout="nchw", out=y))
    elif args.ops_only == "backward":
        xn = torch.from_numpy(workloads.workload_nchw_512(seed=5).astype(np.float32)).to(dev)
        ops = []
        for method in ("bilinear", "bicubic"):
            for s in (2.0, 0.5):
                Ho = int(512 * s)
                g = torch.randn((32, 3, Ho, Ho), dtype=torch.float32, device=dev)
                gi = torch.empty_like(xn)
                ws = torch.empty(rs.backward_workspace_bytes(g, (512, 512), method), dtype=torch.uint8, device=dev)
                ops.append(lambda g=g, gi=gi, ws=ws, m=method: rs.resize_backward(g, (512, 512), m, grad_in=gi,
                                                                                 workspace=ws))
    elif args.ops_only == "rgb":
        img = workloads.workload_rgb_4096(seed=2)
        x = torch.from_numpy(img).to(dev)
        ops = []
        for _, method, s in RGB_OPS:
            Ho = out_hw(4096, s)
            y = torch.empty((Ho, Ho, 3), dtype=torch.uint8, device=dev)
            ops.append(lambda y=y, m=method, Ho=Ho: rs.resize(x, (Ho, Ho), m, out=y))
    elif args.ops_only == "sweep":
        x = torch.from_numpy(workloads.uniform_u8(6, 800, 800, 1)).to(dev)
        y = torch.empty((3200, 3200, 1), dtype=torch.uint8, device=dev)
        ops = [lambda t=t: rs.resize(x, (3200, 3200), "bilinear", out=y, impl="plain", tile=t) for t in ((32, 4), (4, 32))]
    elif args.ops_only == "serving":
        frames = torch.from_numpy(np.stack([workloads.smooth_field_u8(600 + k, 1080, 1920, 3) for k in range(16)])).to(dev)
        y8 = torch.empty((16, 224, 398, 3), dtype=torch.uint8, device=dev)
        yh = torch.empty((16, 3, 256, 455), dtype=torch.float16, device=dev)
        mean_t, std_t = (123.675, 116.28, 103.53), (58.395, 57.12, 57.375)
        ops = [lambda: rs.resize(frames, (224, 398), "bicubic", out=y8, antialias=True),
               lambda: rs.resize_normalize(frames, (256, 455), "bilinear", mean_t, std_t, dtype=torch.float16, out=yh,
                                           antialias=True)]
    elif args.ops_only == "float":
        f64 = workloads.workload_float_8192(seed=3)
        ops = []
        for tdt in (torch.float32, torch.float16, torch.bfloat16):
            xf = torch.from_numpy(f64).to(dev).to(tdt)
            yf = torch.empty((16384, 16384), dtype=tdt, device=dev)
            ops.append(lambda xf=xf, yf=yf: rs.resize(xf, (16384, 16384), "bicubic", out=yf))
    else:
        b = Batch(torch, workloads, dev, args.batch_images)
        if not args.no_autotune:   # the item shape the timed plan uses
            rs.autotune_batched(b.srcs, b.outs, b.methods)
        plan = rs.BatchedPlan(b.srcs, b.outs, b.methods)
        ops = [plan.launch]
    flush = Flusher(torch, dev) if args.flush_between else None
    torch.cuda.synchronize()
    # the launches below, alone, under `ncu --profile-from-start off`
    torch.cuda.profiler.start()
    for _ in range(args.warmup + args.steps):
        for fn in ops:
            fn()
            if flush:
                flush()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


def run_ours(args, rank, world, local):
    import torch
    import paper_1001_1718_gb300 as rs
    from paper_1001_1718_gb300 import workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream(dev)

    if args.ops_only:
        profile_ops(args, torch, rs, workloads, dev)
        return None

    b = Batch(torch, workloads, dev)
    tuned = None
    if not args.no_autotune:   # outside the timed region; cached for the plan below
        tuned = rs.autotune_batched(b.srcs, b.outs, b.methods)
    plan = rs.BatchedPlan(b.srcs, b.outs, b.methods)
    kernels = plan.kernels()
    flush = Flusher(torch, dev)

    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = time_ops(torch, stream, [("batch", plan.launch)], args.steps, args.warmup, flush)["batch"]
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()

    px_per_s, total_s = aggregate(b.out_px, args.steps, sum(times) / 1e3, world)
    value = px_per_s / 1e9
    assert rs.debug_fault() == 0, "a kernel reported a bound violation"

    # Roofline of the step's one launch (the plan): algorithmic bytes = every
    # source read once + every output written once.
    mean_ms = statistics.mean(times)
    alg_bytes = b.in_bytes + b.out_bytes
    achieved = alg_bytes / (mean_ms / 1e3) / 1e9
    traffic = traffic_from_profile("k_batched_window", "batch256")

    e2e = run_e2e_batch(torch, rs, b, plan, dev, stream, min(args.steps, 10), 2)

    line = {
        "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "images": len(b.items), "storage": "u8 HWC interleaved, C=3",
                   "coord": "asymmetric (Eq. 1)", "cubic_a": -0.5,
                   "kernel": f"replayable batch plan: {kernels} persistent class launches in one CUDA graph",
                   "item_shape": ({"autotuned": True, **tuned} if tuned else {"autotuned": False}),
                   "l2": "flushed before every timed step (256 MB write); step I/O 6.6 GB",
                   "parallelism": f"replicas x{world} (each GPU its own batch)",
                   "output_px_per_step": b.out_px, "in_bytes_per_step": b.in_bytes,
                   "out_bytes_per_step": b.out_bytes},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "kernel": f"the batch plan ({kernels} k_batched_window / k_batched class launches, one graph)",
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": f"{peak_kind} copy bandwidth"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": kernels * args.steps,
    }
    if rank == 0:
        from oracle import oracle
        oracle.build()
        line["error"] = batch_errors(oracle, b, b.outs)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(oracle, b, budget_s=8.0)
        if not args.no_extras:
            line["extras"] = extras(torch, rs, dev, stream, oracle, hbm_peak, b)
    plan.close()
    return line


def run_e2e_batch(torch, rs, b, plan, dev, stream, steps, warmup):
    """The batch end to end through the public API with host buffers: every
    step copies the 256 inputs from pinned host memory, replays a plan and
    copies the 256 outputs back to pinned host memory. Two sets of device
    outputs (two plans over the same inputs) alternate between steps, so a
    step's outputs go back on a copy stream while the next step's inputs come
    in and its plan runs; a plan waits only until its own output set has been
    read back (two steps earlier), and a step's input copies wait for the
    previous plan on the same stream."""
    host_in = [torch.from_numpy(im).pin_memory() for im in b.imgs]
    host_out = [torch.empty(y.shape, dtype=y.dtype, pin_memory=True) for y in b.outs]
    outs2 = [torch.empty_like(y) for y in b.outs]
    plans = [plan, rs.BatchedPlan(b.srcs, outs2, b.methods)]
    out_sets = [b.outs, outs2]
    copy_stream = torch.cuda.Stream(dev)
    ev_plan = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    for e in ev_out:
        e.record(copy_stream)
    k = [0]

    def step():
        i = k[0] % 2
        k[0] += 1
        with torch.cuda.stream(stream):
            for h, d in zip(host_in, b.srcs):
                d.copy_(h, non_blocking=True)
            stream.wait_event(ev_out[i])
            plans[i].launch()
            ev_plan[i].record(stream)
        copy_stream.wait_event(ev_plan[i])
        with torch.cuda.stream(copy_stream):
            for d, h in zip(out_sets[i], host_out):
                h.copy_(d, non_blocking=True)
            ev_out[i].record(copy_stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    stream.wait_event(ev_out[0])   # the timed region ends when every output has landed
    stream.wait_event(ev_out[1])
    e.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / steps
    plans[1].close()
    del outs2
    return {"value": b.out_px / (ms / 1e3) / 1e9, "unit": "Gpixels/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(b.in_bytes), "d2h_bytes_per_step": int(b.out_bytes),
            "note": "pinned host buffers; two device output sets alternate between steps; bound by the "
                    "device-to-host link"}


def _oracle_batch_sample(oracle, b, budget_s, band=16, every=16, max_steps=None):
    """The FP64 oracle on bands of `band` output rows of every `every`-th
    batch image, round robin, until `budget_s` seconds of wall time (or
    max_steps bands) have been spent."""
    picks = list(range(0, len(b.items), every))
    if not hasattr(b, "f64"):
        b.f64 = {}   # FP64 copies of the sampled images, made once
    f64 = b.f64
    px, k = 0, 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s and (max_steps is None or k < max_steps):
        idx = picks[k % len(picks)]
        it = b.items[idx]
        if idx not in f64:
            f64[idx] = b.imgs[idx].astype(np.float64)
        nb = min(band, it.Ho)
        y0 = (k * 131) % max(1, it.Ho - nb + 1)
        ys = np.repeat(np.arange(y0, y0 + nb), it.Wo)
        xs = np.tile(np.arange(it.Wo), nb)
        oracle.resize_points(f64[idx], it.Ho, it.Wo, it.method, 0, -0.5, ys, xs)
        px += len(ys)
        k += 1
    dt = time.perf_counter() - t0
    return px, dt, k, len(picks)


def cpu_baseline(oracle, b, budget_s=8.0, single_s=2.0):
    """The FP64 oracle on this host's cores on a bounded sample of the batch
    step (bands of output rows of 16 of its images), then the same on one
    thread (reported beside it)."""
    px, dt, k, npk = _oracle_batch_sample(oracle, b, budget_s)
    line = {"value": px / dt / 1e9, "unit": "Gpixels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} bands of 16 output rows round robin over {npk} of the 256 batch images "
                      f"({px} output px, {dt:.1f} s wall)"}
    if single_s > 0:
        cores = oracle.num_threads()
        oracle.set_num_threads(1)
        try:
            px1, dt1, k1, _ = _oracle_batch_sample(oracle, b, single_s)
        finally:
            oracle.set_num_threads(cores)
        line["single_thread"] = {"value": px1 / dt1 / 1e9, "unit": "Gpixels/s", "cores": 1,
                                 "sample": f"{k1} bands ({px1} output px, {dt1:.1f} s wall)"}
    return line


# --------------------------------------------------------------------------
# Extra configurations

def extras(torch, rs, dev, stream, oracle, hbm_peak, b):
    from paper_1001_1718_gb300 import workloads
    ex = {}
    flush = Flusher(torch, dev)

    def bench(fn, reps=20):
        t = time_ops(torch, stream, [("op", fn)], reps, 3, flush)["op"]
        return statistics.median(t)

    def rec(name, ms, in_bytes, out_bytes, out_px, **kw):
        gbs = (in_bytes + out_bytes) / (ms / 1e3) / 1e9
        ex[name] = {"ms": ms, "gpx_s": out_px / (ms / 1e3) / 1e9, "hbm_gbs": gbs,
                    "frac_of_hbm_peak": gbs / hbm_peak, **kw}
        return ex[name]

    # --- the batch beside it: one launch per image (AUTO), and the paper's
    # plain kernel (one thread per output pixel, 32x4 blocks) on FP32 copies
    def per_image():
        for x, y, m in zip(b.srcs, b.outs, b.methods):
            rs.resize(x, y.shape[:2], m, out=y)
    ms = bench(per_image, 5)
    rec("batch256_u8_one_launch_per_image", ms, b.in_bytes, b.out_bytes, b.out_px, launches=len(b.items))
    x32 = [x.float() for x in b.srcs]
    y32 = [torch.empty(y.shape, dtype=torch.float32, device=dev) for y in b.outs]

    def plain_all():
        for x, y, m in zip(x32, y32, b.methods):
            rs.resize(x, y.shape[:2], m, out=y, impl="plain")
    ms = bench(plain_all, 3)
    rec("batch256_f32_plain_kernel", ms, 4 * b.in_bytes, 4 * b.out_bytes, b.out_px, launches=len(b.items),
        note="the paper's kernel (Sec. III.A, Eq. 6; 32x4 blocks) on FP32 copies of the batch",
        error=batch_errors(oracle, b, y32, "f32"))
    del x32, y32
    torch.cuda.empty_cache()

    # --- RGB uint8 4096x4096: bicubic x2, bicubic x1.7, nearest x2 (AUTO),
    # with the roofline of its dominant launch (the exact-x2 window kernel)
    img = workloads.workload_rgb_4096(seed=2)
    x = torch.from_numpy(img).to(dev)
    outs = {}
    ops = []
    for name, method, s in RGB_OPS:
        Ho = out_hw(4096, s)
        y = torch.empty((Ho, Ho, 3), dtype=torch.uint8, device=dev)
        outs[name] = (y, rs.METHODS[method])
        ops.append((name, (lambda y=y, m=method, Ho=Ho: rs.resize(x, (Ho, Ho), m, out=y))))
    times = time_ops(torch, stream, ops, 50, 5, flush)
    step_ms = [sum(times[n][k] for n, _ in ops) for k in range(50)]
    px = sum(y.shape[0] * y.shape[1] for y, _ in outs.values())
    per_op = {}
    for n, _ in ops:
        ms = statistics.mean(times[n])
        byt = img.size + outs[n][0].numel()
        per_op[n] = {"ms": ms, "gpx_s": outs[n][0].shape[0] * outs[n][0].shape[1] / (ms / 1e3) / 1e9,
                     "hbm_gbs": byt / (ms / 1e3) / 1e9, "frac_of_hbm_peak": byt / (ms / 1e3) / 1e9 / hbm_peak}
    chosen = rs.tile_config(x, (8192, 8192), "bicubic")
    kname = KERNEL_NAMES.get(chosen["impl"], chosen["impl"])
    errs = {}
    x64 = img.astype(np.float64)
    for n, (y, code) in outs.items():
        ys, xs = workloads.sample_points(7, y.shape[0], y.shape[1], 4096)
        ref = oracle.resize_points(x64, y.shape[0], y.shape[1], code, 0, -0.5, ys, xs)
        got = y[torch_index(ys), torch_index(xs)].cpu().numpy().astype(np.float64)
        errs[n] = {"max_abs_vs_f64": float(np.abs(got - ref).max()), "mean_abs_vs_f64": float(np.abs(got - ref).mean()),
                   "max_steps_vs_rounded_oracle": float(np.abs(got - oracle.quantize_u8(ref)).max())}
    bc = per_op["bicubic_x2"]
    ex["rgb4096_u8_step"] = {
        "ms": statistics.mean(step_ms), "gpx_s": px / (statistics.mean(step_ms) / 1e3) / 1e9, "per_op": per_op,
        "error_sampled_4096_points": errs,
        "roofline": {"bound": "hbm", "achieved": bc["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                     "frac": bc["frac_of_hbm_peak"], "traffic": traffic_from_profile(kname, "rgb4096_bicubic_x2"),
                     "kernel": f"{kname}<bicubic, C=3, u8> exact x2 ({chosen})",
                     "algorithmic_bytes_per_launch": img.size + 8192 * 8192 * 3}}
    ms = bench(lambda: rs.resize(x, (8192, 8192), "bicubic", out=outs["bicubic_x2"][0], impl="plain"), 10)
    rec("rgb4096_u8_bicubic_x2_plain_kernel", ms, img.size, 8192 * 8192 * 3, 8192 * 8192)
    del x, outs, ops
    torch.cuda.empty_cache()

    # --- single-channel 8192x8192 field, bicubic x2, stored as FP32 / FP16 / BF16
    f64 = workloads.workload_float_8192(seed=3)
    Hf, Wf = f64.shape
    ys, xs = workloads.sample_points(3, 2 * Hf, 2 * Wf, 2048)
    ref_true = oracle.resize_points(f64, 2 * Hf, 2 * Wf, 2, 0, -0.5, ys, xs)[:, 0]
    for dt_name, tdt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
        xf = torch.from_numpy(f64).to(dev).to(tdt)
        yf = torch.empty((2 * Hf, 2 * Wf), dtype=tdt, device=dev)
        stored64 = xf.to(torch.float64).cpu().numpy()
        ref = oracle.resize_points(stored64, 2 * Hf, 2 * Wf, 2, 0, -0.5, ys, xs)[:, 0]
        for impl in (("auto", "plain") if dt_name == "f32" else ("auto",)):
            ms = bench(lambda: rs.resize(xf, (2 * Hf, 2 * Wf), "bicubic", out=yf, impl=impl), 10)
            got = yf[torch_index(ys), torch_index(xs)].to(torch.float64).cpu().numpy()
            es = xf.element_size()
            rec(f"float8192_bicubic_x2_{dt_name}_{impl}", ms, Hf * Wf * es, 4 * Hf * Wf * es, 4 * Hf * Wf,
                max_abs_vs_f64_of_stored_input=float(np.abs(got - ref).max()),
                mean_abs_vs_f64_of_stored_input=float(np.abs(got - ref).mean()),
                max_abs_vs_f64_of_fp64_input=float(np.abs(got - ref_true).max()),
                mean_abs_vs_f64_of_fp64_input=float(np.abs(got - ref_true).mean()))
        del xf, yf
    torch.cuda.empty_cache()

    # --- uint8 512x512 bilinear x2 (L2-resident, launch-bound): device time
    # of a direct launch, and of one replay of a CUDA graph holding the call
    img1, (Ho, Wo) = workloads.workload_u8_bilinear_512(seed=1)
    x1 = torch.from_numpy(img1).to(dev)
    y1 = torch.empty((Ho, Wo, 1), dtype=torch.uint8, device=dev)
    ref1 = oracle.quantize_u8(oracle.resize(img1.astype(np.float64), Ho, Wo, 1))
    for impl in ("auto", "plain"):
        ms = bench(lambda: rs.resize(x1, (Ho, Wo), "bilinear", out=y1, impl=impl), 50)
        rec(f"u8_512_bilinear_x2_{impl}", ms, img1.size, y1.numel(), Ho * Wo,
            bit_exact_vs_oracle=bool(np.array_equal(y1.cpu().numpy(), ref1)),
            note="L2-resident: roofline fraction not meaningful")
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        rs.resize(x1, (Ho, Wo), "bilinear", out=y1)   # warm the library's per-kernel caches
    side.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        rs.resize(x1, (Ho, Wo), "bilinear", out=y1)
    y1.zero_()
    ms = bench(graph.replay, 50)
    reps = 200
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        graph.replay()
    e.record(stream)
    torch.cuda.synchronize()
    rec("u8_512_bilinear_x2_graph_replay", ms, img1.size, y1.numel(), Ho * Wo,
        back_to_back_us_per_replay=a.elapsed_time(e) * 1e3 / reps,
        bit_exact_vs_oracle=bool(np.array_equal(y1.cpu().numpy(), ref1)),
        note="one replay of a CUDA graph holding the resize (device time, L2 flushed before)")
    del graph

    # --- the fused serving pre-process (resample + per-channel normalise +
    # HWC uint8 -> planar FP16) against the unfused path: the library's
    # uint8 resize, then torch's permute / normalise / cast
    mean_t, std_t = (123.675, 116.28, 103.53), (58.395, 57.12, 57.375)
    for name, (N, H, W), (Ho, Wo), method, aa in (
            ("frames32_1024_to_512_bilinear", (32, 1024, 1024), (512, 512), "bilinear", False),
            ("frames32_512_to_1024_bicubic", (32, 512, 512), (1024, 1024), "bicubic", False),
            ("frames16_1080p_to_256x455_bilinear", (16, 1080, 1920), (256, 455), "bilinear", False),
            ("frames16_1080p_to_256x455_bilinear_antialias", (16, 1080, 1920), (256, 455), "bilinear", True),
            ("frames16_1080p_to_224x398_bicubic_antialias", (16, 1080, 1920), (224, 398), "bicubic", True)):
        frames = np.stack([workloads.smooth_field_u8(600 + k, H, W, 3) for k in range(N)])
        xf = torch.from_numpy(frames).to(dev)
        yo = torch.empty((N, 3, Ho, Wo), dtype=torch.float16, device=dev)
        try:
            rs.resize_normalize(xf, (Ho, Wo), method, mean_t, std_t, dtype=torch.float16, out=yo, antialias=aa)
        except rs.ResampleError as e:
            ex[f"normalize_{name}"] = {"unsupported": str(e)}
            continue
        ms_f = bench(lambda: rs.resize_normalize(xf, (Ho, Wo), method, mean_t, std_t, dtype=torch.float16, out=yo,
                                                 antialias=aa), 20)
        yu8 = torch.empty((N, Ho, Wo, 3), dtype=torch.uint8, device=dev)
        mt = torch.tensor(mean_t, device=dev).view(1, 3, 1, 1)
        st = torch.tensor(std_t, device=dev).view(1, 3, 1, 1)

        def unfused():
            rs.resize(xf, (Ho, Wo), method, out=yu8, antialias=aa)
            torch.sub(yu8.permute(0, 3, 1, 2).float(), mt).div_(st).to(torch.float16)
        ms_u = bench(unfused, 20)
        k0 = 0
        ys, xs = workloads.sample_points(5, Ho, Wo, 2048)
        if aa:
            ref = ((oracle.resize_aa(frames[k0].astype(np.float64), Ho, Wo, rs.METHODS[method]) -
                    np.array(mean_t)) / np.array(std_t)).transpose(2, 0, 1)
        else:
            ref = oracle.resize_normalize(frames[k0].astype(np.float64), Ho, Wo, rs.METHODS[method], mean_t, std_t)
        got = yo[k0][:, torch_index(ys), torch_index(xs)].double().cpu().numpy()
        refp = ref[:, ys, xs]
        unf = ((yu8[k0].permute(2, 0, 1).double() - mt[0].double()) / st[0].double())[:, torch_index(ys), torch_index(xs)]
        rec(f"normalize_{name}_fused_f16", ms_f, xf.numel(), yo.numel() * 2, N * Ho * Wo,
            unfused_ms=ms_u, speedup_vs_unfused=ms_u / ms_f,
            max_abs_vs_f64=float(np.abs(got - refp).max()),
            unfused_max_abs_vs_f64_before_f16=float(np.abs(unf.cpu().numpy() - refp).max()),
            note="one pass: uint8 HWC in, FP16 NCHW out; unfused: uint8 resize, then permute / normalise / cast" +
                 ("; antialiased (the stretched filter; more than 8 taps per axis run the many-tap kernel)" if aa else ""))
        del xf, yo, yu8
    torch.cuda.empty_cache()

    # --- NCHW FP32 32x3x512x512: forward and backward, x2 and x0.5
    xn = torch.from_numpy(workloads.workload_nchw_512(seed=5).astype(np.float32)).to(dev)
    for method in ("bilinear", "bicubic"):
        for s in (2.0, 0.5):
            Ho = Wo = int(512 * s)
            y = torch.empty((32, 3, Ho, Wo), dtype=torch.float32, device=dev)
            ms = bench(lambda: rs.resize(xn, (Ho, Wo), method, layout="nchw", out=y), 10)
            rec(f"nchw_f32_{method}_x{s:g}_fwd", ms, xn.numel() * 4, y.numel() * 4, 96 * Ho * Wo)
            g = torch.randn_like(y)
            gi = torch.empty_like(xn)
            ws = torch.empty(rs.backward_workspace_bytes(g, (512, 512), method), dtype=torch.uint8, device=dev)
            ms = bench(lambda: rs.resize_backward(g, (512, 512), method, grad_in=gi, workspace=ws), 10)
            gp = g[0, 0].cpu().numpy().astype(np.float64)
            ref = oracle.adjoint(gp, 512, 512, rs.METHODS[method])[:, :, 0]
            rec(f"nchw_f32_{method}_x{s:g}_bwd", ms, y.numel() * 4, xn.numel() * 4, 96 * 512 * 512,
                max_abs_vs_f64_adjoint_plane0=float(np.abs(gi[0, 0].cpu().numpy() - ref).max()))
            if s < 1:   # antialiased downscale (the filter stretched by the factor)
                ms = bench(lambda: rs.resize(xn, (Ho, Wo), method, layout="nchw", out=y, antialias=True), 10)
                ref = oracle.resize_aa(xn[0, 0].cpu().numpy().astype(np.float64), Ho, Wo,
                                       rs.METHODS[method])[:, :, 0]
                rec(f"nchw_f32_{method}_x{s:g}_fwd_antialias", ms, xn.numel() * 4, y.numel() * 4, 96 * Ho * Wo,
                    max_abs_vs_f64_plane0=float(np.abs(y[0, 0].cpu().numpy() - ref).max()))
            del y, g, gi, ws
    del xn
    torch.cuda.empty_cache()
    return ex


# --------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on this host's cores

class _HostBatch:
    """The batch's host side only (no device)."""

    def __init__(self, workloads):
        self.items = workloads.batch_spec(seed=4)
        every = 16
        self.imgs = [workloads.smooth_field_u8(it.seed, it.H, it.W, 3) if k % every == 0 else None
                     for k, it in enumerate(self.items)]


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import oracle
    from paper_1001_1718_gb300 import workloads
    oracle.build()
    hb = _HostBatch(workloads)
    per_step = 32   # bands of 16 output rows per step

    for idx in range(0, len(hb.items), 16):   # the FP64 copies, before any step
        hb.f64 = getattr(hb, "f64", {})
        hb.f64[idx] = hb.imgs[idx].astype(np.float64)
    for k in range(args.warmup):
        _oracle_batch_sample(oracle, hb, 1e9, max_steps=per_step)
    px, dt, bands, npk = 0, 0.0, 0, 0
    for k in range(args.steps):
        p, d, nb, npk = _oracle_batch_sample(oracle, hb, 1e9, max_steps=per_step)
        px, dt, bands = px + p, dt + d, bands + nb
    value = px / dt / 1e9
    sample = (f"each step: {per_step} bands of 16 output rows of the batch images, round robin over {npk} of "
              f"the 256 images ({px // max(1, args.steps)} output px per step)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(1, args.steps) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "images": 256, "storage": "u8 HWC interleaved, C=3",
                       "coord": "asymmetric (Eq. 1)", "cubic_a": -0.5,
                       "kernel": "FP64 CPU oracle (direct per-pixel loops, OpenMP over points)"},
            "cpu_baseline": {"value": value, "unit": "Gpixels/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gpixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def tile_sweep():
    """The tiling study of the paper (Sec. IV-V: one thread per output pixel,
    the block shape decides the time) replayed on this GPU: 800x800 uint8
    single-channel source from the uniform generator, bilinear x2..x10 with
    the plain kernel over block shapes, and the AUTO kernel beside it.
    Median of 20 CUDA-event timed launches, L2 flushed before each."""
    import torch
    import paper_1001_1718_gb300 as rs
    from paper_1001_1718_gb300 import workloads
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = Flusher(torch, dev)
    img = workloads.uniform_u8(6, 800, 800, 1)
    x = torch.from_numpy(img).to(dev)
    shapes = [(32, 4), (4, 32), (16, 8), (8, 16), (8, 8), (16, 16), (32, 8), (64, 4), (128, 1), (32, 32)]
    scales = (2, 4, 6, 8, 10)
    rows = {}
    for sc in scales:
        n = 800 * sc
        y = torch.empty((n, n, 1), dtype=torch.uint8, device=dev)
        for (bw, bh) in shapes + [(0, 0)]:   # (0, 0): AUTO
            impl = "plain" if bw else "auto"
            fn = (lambda: rs.resize(x, (n, n), "bilinear", out=y, impl="plain", tile=(bw, bh))) if bw else \
                 (lambda: rs.resize(x, (n, n), "bilinear", out=y))
            t = time_ops(torch, stream, [("op", fn)], 20, 3, flush)["op"]
            rows.setdefault((bw, bh) if bw else "auto", {})[sc] = statistics.median(t)
    out = ["| kernel / block (w x h) | " + " | ".join(f"x{sc} ({800 * sc}^2) us" for sc in scales) + " |",
           "|---|" + "---|" * len(scales)]
    for key, d in rows.items():
        name = "AUTO (" + rs.tile_config(x, (1600, 1600), "bilinear")["impl"] + " at x2)" if key == "auto" \
            else f"plain {key[0]}x{key[1]}"
        best = {sc: min(rows[k][sc] for k in rows if k != "auto") for sc in scales}
        cells = []
        for sc in scales:
            v = d[sc] * 1e3
            mark = " **best plain**" if key != "auto" and d[sc] == best[sc] else ""
            cells.append(f"{v:.1f}{mark}")
        out.append(f"| {name} | " + " | ".join(cells) + " |")
    print("\n".join(out))


def main():
    args = parse()
    if args.tile_sweep:
        tile_sweep()
        return
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", args.gpus))
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line))
        return
    rank, world, local = dist_init(args.gpus)
    line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
