"""Benchmark of the resampling hot path on GB300.

One step = the RGB uint8 4096x4096 smooth-field workload resampled three
ways, each through the C ABI with the tiled kernel:
    bicubic x2   -> 8192 x 8192
    bicubic x1.7 -> 6963 x 6963
    nearest x2   -> 8192 x 8192
value = output pixels per step (an RGB pixel counts once) / device time of
the step, in Gpixels/s, whole job over all ranks. L2 is flushed (a 256 MB
write) before every timed step, outside the step's events.

Extra configurations (measured in the same run, reported under "extras"):
uint8 bilinear 512x512 x2; float 8192x8192 bicubic x2 stored as FP32 / FP16 /
BF16; the plain one-thread-per-pixel kernel on the same problems; NCHW FP32
forward + backward; the ragged 256-image batch.

--impl reference times the FP64 CPU oracle on the same workload (bounded
sample per step) on this host's cores.
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
HEADLINE_OPS = (("bicubic_x2", "bicubic", 2.0), ("bicubic_x1.7", "bicubic", 1.7), ("nearest_x2", "nearest", 2.0))
FALLBACK_HBM_GBS = 6800.0
KERNEL_NAMES = {"window": "k_win", "stream": "k_stream", "tiled": "k_tiled", "gather": "k_nearest",
                "plain": "k_plain"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="tune tile shapes before timing")
    ap.add_argument("--tile-sweep", action="store_true",
                    help="the paper's tiling experiment on this GPU: an 800x800 uint8 image, bilinear at scales "
                         "2..10, the paper's kernel (one thread per output pixel) over block shapes, against "
                         "AUTO; prints a markdown table and exits")
    ap.add_argument("--ops-only", nargs="?", const="headline", default=None,
                    choices=["headline", "nchw", "backward", "batch"],
                    help="profiling driver: run warmup + steps of the three headline resizes (headline), "
                         "of the NCHW FP32 forward or backward x2 / x0.5 (nchw, backward) or of the "
                         "256-image batch plan (batch), and exit")
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


def sample_errors(oracle, img64, outs, methods, seed=0, n=4096):
    """max / mean |gpu - FP64 oracle| on n sampled output points per op."""
    from paper_1001_1718_gb300 import workloads
    res = {}
    for name, (y, code) in outs.items():
        Ho, Wo = y.shape[0], y.shape[1]
        ys, xs = workloads.sample_points(seed, Ho, Wo, n)
        ref = oracle.resize_points(img64, Ho, Wo, code, 0, -0.5, ys, xs)
        got = y[torch_index(ys), torch_index(xs)].cpu().numpy().astype(np.float64)
        q = oracle.quantize_u8(ref).astype(np.float64)
        res[name] = {"max_abs_vs_f64": float(np.abs(got - ref).max()),
                     "mean_abs_vs_f64": float(np.abs(got - ref).mean()),
                     "max_steps_vs_rounded_oracle": float(np.abs(got - q).max()),
                     "points": int(n)}
    return res


def torch_index(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.int64)).cuda()


def profile_ops(args, torch, rs, workloads, dev):
    """Untimed launches for profiling under ncu: the NCHW FP32 forward or
    backward (bilinear / bicubic, x2 and x0.5 of 32x3x512x512) or the
    replayable plan of the 256-image ragged batch."""
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
    else:
        items = workloads.batch_spec(seed=4)
        srcs = [torch.from_numpy(im).to(dev) for im in workloads.batch_images(items)]
        outs = [torch.empty((it.Ho, it.Wo, 3), dtype=torch.uint8, device=dev) for it in items]
        plan = rs.BatchedPlan(srcs, outs, [workloads.METHOD_NAMES[it.method] for it in items])
        ops = [plan.launch]
    for _ in range(args.warmup + args.steps):
        for fn in ops:
            fn()
    torch.cuda.synchronize()


def run_ours(args, rank, world, local):
    import torch
    import paper_1001_1718_gb300 as rs
    from paper_1001_1718_gb300 import workloads

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hbm_peak, peak_kind = peaks()
    stream = torch.cuda.current_stream(dev)

    if args.ops_only in ("nchw", "backward", "batch"):
        profile_ops(args, torch, rs, workloads, dev)
        return None

    img = workloads.workload_rgb_4096(seed=2)
    H, W, C = img.shape
    x = torch.from_numpy(img).to(dev)
    outs = {}
    ops = []
    for name, method, s in HEADLINE_OPS:
        Ho, Wo = out_hw(H, s), out_hw(W, s)
        y = torch.empty((Ho, Wo, C), dtype=torch.uint8, device=dev)
        outs[name] = (y, rs.METHODS[method])
        if args.autotune:
            rs.autotune(x, (Ho, Wo), method, out=y)
        ops.append((name, (lambda y=y, m=method, Ho=Ho, Wo=Wo: rs.resize(x, (Ho, Wo), m, out=y))))
    px_per_step = sum(y.shape[0] * y.shape[1] for y, _ in outs.values())
    if args.ops_only:
        for _ in range(args.warmup + args.steps):
            for _, fn in ops:
                fn()
        torch.cuda.synchronize()
        return None
    flush = Flusher(torch, dev)

    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = time_ops(torch, stream, ops, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()

    step_ms = [sum(times[n][s] for n, _ in ops) for s in range(args.steps)]
    px_per_s, total_s = aggregate(px_per_step, args.steps, sum(step_ms) / 1e3, world)
    value = px_per_s / 1e9
    assert rs.debug_fault() == 0, "a kernel reported a bound violation"

    # Roofline of the dominant kernel (bicubic x2): algorithmic bytes = source
    # read once + output written once.
    bc_ms = statistics.mean(times["bicubic_x2"])
    Ho2, Wo2 = outs["bicubic_x2"][0].shape[:2]
    alg_bytes = H * W * C + Ho2 * Wo2 * C
    achieved = alg_bytes / (bc_ms / 1e3) / 1e9
    chosen = rs.tile_config(x, (Ho2, Wo2), "bicubic")
    kname = KERNEL_NAMES.get(chosen["impl"], chosen["impl"])
    traffic = traffic_from_profile(kname, "rgb4096_bicubic_x2")
    per_op = {n: {"ms": statistics.mean(times[n]),
                  "gpx_s": outs[n][0].shape[0] * outs[n][0].shape[1] / (statistics.mean(times[n]) / 1e3) / 1e9,
                  "hbm_gbs": (H * W * C + outs[n][0].numel()) / (statistics.mean(times[n]) / 1e3) / 1e9}
              for n, _ in ops}
    for n in per_op:
        per_op[n]["frac_of_hbm_peak"] = per_op[n]["hbm_gbs"] / hbm_peak

    # End to end through the public API with host buffers: H2D of the input
    # from pinned memory, the three resizes, D2H of the three outputs.
    e2e = run_e2e(torch, rs, img, outs, dev, stream, min(args.steps, 20), 3)

    line = {
        "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "rgb_u8_4096x4096_smooth_field: bicubic x2, bicubic x1.7, nearest x2",
                   "storage": "u8 HWC interleaved, C=3", "coord": "asymmetric (Eq. 1)", "cubic_a": -0.5,
                   "kernel": "library default per op (rs_resize_ex, RS_IMPL_AUTO)",
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"replicas x{world} (independent images per GPU)",
                   "output_px_per_step": px_per_step},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "kernel": f"{kname}<bicubic, C=3, u8> bicubic x2 ({chosen})",
                     "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": f"{peak_kind} copy bandwidth"},
        "per_op": per_op,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": len(ops) * args.steps,
    }
    if rank == 0:
        from oracle import oracle
        oracle.build()
        line["error"] = sample_errors(oracle, img.astype(np.float64), outs, None)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(oracle, img, budget_s=8.0)
        if not args.no_extras:
            line["extras"] = extras(torch, rs, dev, stream, oracle, hbm_peak)
    return line


def run_e2e(torch, rs, img, outs, dev, stream, steps, warmup):
    host_in = torch.from_numpy(img).pin_memory()
    host_out = {n: torch.empty(y.shape, dtype=y.dtype).pin_memory() for n, (y, _) in outs.items()}
    dev_in = torch.empty(img.shape, dtype=torch.uint8, device=dev)
    names = [n for n, _, _ in HEADLINE_OPS]
    meth = {n: m for n, m, _ in HEADLINE_OPS}

    # Each output's device-to-host copy runs on a copy stream as soon as its
    # resize is done, overlapping the next resizes and the next step's
    # host-to-device copy; a resize waits until the previous copy of its
    # output buffer has finished.
    copy_stream = torch.cuda.Stream(dev)
    ev_k = {n: torch.cuda.Event() for n in names}
    ev_c = {n: torch.cuda.Event() for n in names}
    for n in names:
        ev_c[n].record(copy_stream)

    def step():
        dev_in.copy_(host_in, non_blocking=True)
        for n in names:
            y = outs[n][0]
            stream.wait_event(ev_c[n])
            rs.resize(dev_in, y.shape[:2], meth[n], out=y)
            ev_k[n].record(stream)
            copy_stream.wait_event(ev_k[n])
            with torch.cuda.stream(copy_stream):
                host_out[n].copy_(y, non_blocking=True)
            ev_c[n].record(copy_stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    for n in names:   # the timed region ends when every copy has landed
        stream.wait_event(ev_c[n])
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    px = sum(outs[n][0].shape[0] * outs[n][0].shape[1] for n in names)
    return {"value": px / (ms / 1e3) / 1e9, "unit": "Gpixels/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(host_in.numel()),
            "d2h_bytes_per_step": int(sum(t.numel() for t in host_out.values()))}


def cpu_baseline(oracle, img, budget_s=8.0, band=64, single_s=2.0):
    """The FP64 oracle on this host's cores on a bounded sample of the step:
    bands of `band` output rows of each of the three outputs, round robin,
    until `budget_s` seconds of wall time have been spent; then the same on
    one thread for `single_s` seconds (reported beside it)."""
    line = _oracle_sample(oracle, img, budget_s, band)
    if single_s > 0:
        cores = oracle.num_threads()
        oracle.set_num_threads(1)
        try:
            one = _oracle_sample(oracle, img, single_s, band)
        finally:
            oracle.set_num_threads(cores)
        line["single_thread"] = {"value": one["value"], "unit": one["unit"], "cores": 1, "sample": one["sample"]}
    return line


def _oracle_sample(oracle, img, budget_s, band):
    x = img.astype(np.float64)
    H, W, C = img.shape
    jobs = []
    for name, method, s in HEADLINE_OPS:
        Ho, Wo = out_hw(H, s), out_hw(W, s)
        code = {"nearest": 0, "bilinear": 1, "bicubic": 2}[method]
        jobs.append((Ho, Wo, code))
    px = 0
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < budget_s:
        Ho, Wo, code = jobs[k % 3]
        y0 = (k * 997 * band) % max(1, Ho - band)
        ys = np.repeat(np.arange(y0, y0 + band), Wo)
        xs = np.tile(np.arange(Wo), band)
        oracle.resize_points(x, Ho, Wo, code, 0, -0.5, ys, xs)
        px += len(ys)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": px / dt / 1e9, "unit": "Gpixels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{k} bands of {band} output rows round robin over bicubic x2 / bicubic x1.7 / nearest x2 "
                      f"({px} output px, {dt:.1f} s wall)"}


# --------------------------------------------------------------------------
# Extra configurations

def extras(torch, rs, dev, stream, oracle, hbm_peak):
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

    # uint8 512x512 bilinear x2 (L2-resident, launch-bound)
    img1, (Ho, Wo) = workloads.workload_u8_bilinear_512(seed=1)
    x1 = torch.from_numpy(img1).to(dev)
    y1 = torch.empty((Ho, Wo, 1), dtype=torch.uint8, device=dev)
    for impl in ("auto", "plain"):
        ms = bench(lambda: rs.resize(x1, (Ho, Wo), "bilinear", out=y1, impl=impl), 50)
        ref = oracle.quantize_u8(oracle.resize(img1.astype(np.float64), Ho, Wo, 1))
        exact = bool(np.array_equal(y1.cpu().numpy(), ref))
        rec(f"u8_512_bilinear_x2_{impl}", ms, img1.size, y1.numel(), Ho * Wo, bit_exact_vs_oracle=exact,
            note="L2-resident: roofline fraction not meaningful")

    # float 8192x8192 bicubic x2 stored as FP32 / FP16 / BF16
    f64 = workloads.workload_float_8192(seed=3)
    Hf, Wf = f64.shape
    ys, xs = workloads.sample_points(3, 2 * Hf, 2 * Wf, 2048)
    for dt_name, tdt in (("f32", torch.float32), ("f16", torch.float16), ("bf16", torch.bfloat16)):
        xf = torch.from_numpy(f64).to(dev).to(tdt)
        yf = torch.empty((2 * Hf, 2 * Wf), dtype=tdt, device=dev)
        stored64 = xf.to(torch.float64).cpu().numpy()
        ref = oracle.resize_points(stored64, 2 * Hf, 2 * Wf, 2, 0, -0.5, ys, xs)[:, 0]
        ref_true = oracle.resize_points(f64, 2 * Hf, 2 * Wf, 2, 0, -0.5, ys, xs)[:, 0]
        for impl in (("auto", "plain") if dt_name == "f32" else ("auto",)):
            ms = bench(lambda: rs.resize(xf, (2 * Hf, 2 * Wf), "bicubic", out=yf, impl=impl), 10)
            got = yf[torch_index(ys), torch_index(xs)].to(torch.float64).cpu().numpy()
            es = xf.element_size()
            rec(f"float_8192_bicubic_x2_{dt_name}_{impl}", ms, Hf * Wf * es, 4 * Hf * Wf * es, 4 * Hf * Wf,
                max_abs_vs_f64_of_stored_input=float(np.abs(got - ref).max()),
                mean_abs_vs_f64_of_stored_input=float(np.abs(got - ref).mean()),
                max_abs_vs_f64_of_fp64_input=float(np.abs(got - ref_true).max()),
                mean_abs_vs_f64_of_fp64_input=float(np.abs(got - ref_true).mean()))
        del xf, yf
    torch.cuda.empty_cache()

    # ragged batch: one persistent launch replayed from a CUDA graph, vs
    # one launch per image
    items = workloads.batch_spec(seed=4)
    imgs = workloads.batch_images(items)
    srcs = [torch.from_numpy(im).to(dev) for im in imgs]
    outs = [torch.empty((it.Ho, it.Wo, 3), dtype=torch.uint8, device=dev) for it in items]
    meths = [workloads.METHOD_NAMES[it.method] for it in items]
    in_b = sum(x.numel() for x in srcs)
    out_b = sum(y.numel() for y in outs)
    out_px = sum(it.Ho * it.Wo for it in items)
    plan = rs.BatchedPlan(srcs, outs, meths)
    ms = bench(lambda: plan.launch(), 10)
    ys, xs = workloads.sample_points(4, items[0].Ho, items[0].Wo, 512)
    errs = []
    for k in (0, 1, 100, 255):
        it = items[k]
        ys, xs = workloads.sample_points(k, it.Ho, it.Wo, 512)
        ref = oracle.resize_points(imgs[k].astype(np.float64), it.Ho, it.Wo, it.method, 0, -0.5, ys, xs)
        got = outs[k][torch_index(ys), torch_index(xs)].cpu().numpy().astype(np.float64)
        errs.append(float(np.abs(got - oracle.quantize_u8(ref)).max()))
    rec("batch256_rgb_u8_graph", ms, in_b, out_b, out_px, images=len(items),
        max_steps_vs_rounded_oracle_sampled=max(errs), launches=1)

    def per_image():
        for x, y, m in zip(srcs, outs, meths):
            rs.resize(x, y.shape[:2], m, out=y)
    ms = bench(per_image, 5)
    rec("batch256_rgb_u8_per_image_launches", ms, in_b, out_b, out_px, images=len(items), launches=len(items))
    plan.close()
    del srcs, outs, plan
    torch.cuda.empty_cache()

    # NCHW FP32 32x3x512x512: forward and backward, x2 and x0.5
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

    # plain kernel on the headline's dominant problem
    img = workloads.workload_rgb_4096(seed=2)
    x = torch.from_numpy(img).to(dev)
    y = torch.empty((8192, 8192, 3), dtype=torch.uint8, device=dev)
    ms = bench(lambda: rs.resize(x, (8192, 8192), "bicubic", out=y, impl="plain"), 10)
    rec("rgb_u8_4096_bicubic_x2_plain", ms, img.size, y.numel(), 8192 * 8192)
    del x, y
    torch.cuda.empty_cache()
    return ex


# --------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on this host's cores

def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import oracle
    from paper_1001_1718_gb300 import workloads
    oracle.build()
    img = workloads.workload_rgb_4096(seed=2)
    x = img.astype(np.float64)
    H, W, C = img.shape
    band = 32
    jobs = []
    for name, method, s in HEADLINE_OPS:
        Ho, Wo = out_hw(H, s), out_hw(W, s)
        jobs.append((Ho, Wo, {"nearest": 0, "bilinear": 1, "bicubic": 2}[method]))

    def step(k):
        px = 0
        for (Ho, Wo, code) in jobs:
            y0 = (k * 131 * band) % (Ho - band)
            ys = np.repeat(np.arange(y0, y0 + band), Wo)
            xs = np.tile(np.arange(Wo), band)
            oracle.resize_points(x, Ho, Wo, code, 0, -0.5, ys, xs)
            px += len(ys)
        return px

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    px = 0
    for k in range(args.steps):
        px += step(k)
    dt = time.perf_counter() - t0
    value = px / dt / 1e9
    sample = (f"each step: {band} output rows of each of bicubic x2, bicubic x1.7, nearest x2 "
              f"({px // max(1, args.steps)} output px per step)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gpixels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "rgb_u8_4096x4096_smooth_field: bicubic x2, bicubic x1.7, nearest x2",
                       "storage": "u8 HWC interleaved, C=3", "coord": "asymmetric (Eq. 1)", "cubic_a": -0.5,
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
