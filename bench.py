"""Benchmark of the Local-GS rasterization path on one GB300 (or N replicas).

Workload (outdoor scene): 500,000 Gaussians FP32 with SH degree 3 drawn from 64
anisotropic clusters plus a 10 % background shell at radius 10, seen by 8
orbit cameras at 1264x832. One step renders all 8 views through the whole hot
path: preprocess -> scan/emit/radix sort/ranges -> render, in one batched
launch per stage, with the tile shape, warp-block layout and staging batch the
autotuner picks. ``value`` is frames (views) per second over all ranks; Mpix/s,
the plain tiled rasterizer on the same inputs, forward + backward, per-stage
times and the roofline of the dominant kernel (against FP32 and SFU peaks
measured on the GPU by the library's probe kernels) are reported beside it,
plus the small (10k), batched (64 views), indoor training and 30M-Gaussian
configurations.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream; a step's time is the median over the K steps. L2 is flushed
(256 MB write) between steps, outside the events. Under torchrun each rank
renders its own 8 views (replicas: no data exchange), and the time is the
maximum over ranks.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (the
reference arm of this project: there is no other implementation to run), one
full view per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "outdoor-500k-sh3-8x1264x832"
METRIC = "frames/s (Local-GS fwd, 8 views of 1264x832, 500k Gaussians SH3)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--tile", default="auto",
                   help="tile shape WxH, or auto: the autotuner's pick for the Local-GS forward "
                        "(with --profile, auto means 16x16)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--profile", action="store_true",
                   help="only run warm-up + steps of the Local-GS pipeline (for ncu), no report")
    p.add_argument("--views", type=int, default=8, help="views of the outdoor workload (profiling)")
    p.add_argument("--mode", default="localgs", choices=["localgs", "plain", "literal", "global"])
    p.add_argument("--no-batched", action="store_true", help="skip the 64-view batched workload")
    p.add_argument("--no-indoor", action="store_true", help="skip the indoor training step")
    p.add_argument("--no-scale", action="store_true", help="skip the 30M-Gaussian scale scene")
    p.add_argument("--backward", action="store_true", help="with --profile: also run the adjoint each step")
    p.add_argument("--tight", action="store_true", help="with --profile: tight-box emission")
    p.add_argument("--scene", default="outdoor", choices=["outdoor", "indoor", "scale", "batched"],
                   help="with --profile: the scene (the others run through batch.Renderer)")
    p.add_argument("--block", default="paper",
                   help="warp block WxH of the Local-GS render with a fixed --tile (paper = full-width strips)")
    p.add_argument("--no-tiny", action="store_true", help="skip the 10k-Gaussian 256x256 configuration")
    p.add_argument("--batch", type=int, default=0, help="with --profile: staging batch of the Local-GS render")
    p.add_argument("--sort", default="rts", choices=["rts", "onesweep"],
                   help="with --profile: radix passes as reduce-then-scan kernels or onesweep kernels")
    return p.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            out, _ = self.proc.communicate(timeout=10)
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle arm
def oracle_views(scene, cams, n, first=0):
    """Seconds the FP64 oracle takes to render n full views (preprocess, sort
    and blend of the whole scene for each), cycling through the cameras."""
    import oracle
    t0 = time.perf_counter()
    for k in range(n):
        oracle.render(scene, cams[(first + k) % len(cams)])
    return time.perf_counter() - t0


def cpu_baseline(scene, cams, budget_s=15.0, label="500k Gaussians"):
    import oracle
    t1 = oracle_views(scene, cams, 1)
    n = max(1, min(len(cams), int(budget_s / max(t1, 1e-3))))
    t = oracle_views(scene, cams, n, first=1)
    W, H = cams[0]["width"], cams[0]["height"]
    return {"value": n / t, "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} full {W}x{H} views (FP64 preprocess, sort and blend of all {label} per view)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2606_16566_gb300 import scenes
    import oracle
    scene, cams = scenes.outdoor()
    oracle_views(scene, cams, args.warmup)
    t = oracle_views(scene, cams, args.steps, first=args.warmup)
    fps = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "one full 1264x832 view per step"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "one full 1264x832 view per step (FP64 preprocess, sort and blend of all "
                                   "500k Gaussians), views cycling through the 8 cameras"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reduce_max_over_ranks(values, world, device=None):
    """The element-wise maximum of per-rank timings over all ranks (identity on
    one rank): the slowest rank decides a step's time."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


# ---------------------------------------------------------------- GPU arm
class Pipeline:
    """Preallocated buffers for repeated batched frames through the C ABI."""

    def __init__(self, g, cams, tile, capacity):
        import torch
        from paper_2606_16566_gb300 import lgs
        self.lgs, self.torch = lgs, torch
        self.g, self.cams, self.tile = g, cams, tile
        self.n = g["means"].shape[0]
        self.m = self.n * len(cams)
        self.carr = lgs.cameras(cams)
        dev = g["means"].device
        self.status = lgs.new_status(dev)
        self.pre = lgs.PreOut.empty(self.m, dev)
        self.capacity = capacity
        self.vals = torch.empty(capacity, dtype=torch.int32, device=dev)
        self.ranges = torch.empty((lgs.n_tiles(cams, lgs.config(tile)), 2), dtype=torch.int32, device=dev)
        self.ws = torch.empty(lgs.sort_workspace_size(self.m, capacity), dtype=torch.uint8, device=dev)
        P = lgs.n_pixels(cams)
        self.rgb = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.T = torch.empty(P, dtype=torch.float32, device=dev)
        self.nc = torch.empty(P, dtype=torch.int32, device=dev)

    def stage_pre(self, cfg):
        self.status.zero_()
        self.lgs.preprocess(self.g, self.cams, cfg, out=self.pre, status=self.status)

    def stage_sort(self, cfg):
        # the render consumes values and tile ranges; the 64-bit keys are not materialised
        self.lgs.sort(self.pre, self.n, self.cams, cfg, self.capacity, None, self.vals, self.ranges,
                      self.ws, self.status, with_keys=False)

    def stage_render(self, cfg):
        self.lgs.render_fwd(self.pre, self.vals, self.ranges, self.cams, cfg, self.rgb, self.T, self.nc,
                            self.status)

    def step(self, cfg):
        self.stage_pre(cfg)
        self.stage_sort(cfg)
        self.stage_render(cfg)

    def setup_backward(self, seed=0):
        """Gradient buffers and a fixed upstream gradient dL/drgb (the shape of an
        L1 loss gradient: +-1/numel), so the backward step runs only our kernels."""
        torch = self.torch
        gen = torch.Generator(device=self.rgb.device).manual_seed(seed)
        sign = torch.randint(0, 2, self.rgb.shape, generator=gen, device=self.rgb.device)
        self.d_rgb = (sign.float() * 2 - 1) / self.rgb.numel()
        self.grads = self.lgs.new_grads(self.g, len(self.cams))

    def stage_backward(self, cfg):
        for k in ("means", "scales", "quats", "opacities", "sh"):
            self.grads[k].zero_()
        self.lgs.render_bwd(self.g, self.cams, cfg, self.pre, self.vals, self.ranges, self.T, self.nc,
                            self.d_rgb, None, self.grads, self.status)

    def launches(self):
        """Kernels of one forward step (as in the ncu launch list): preprocess;
        4 entry passes of 3 kernels (upsweep, scan, downsweep; the first forms
        the depth keys); gather or tight count (folded into the last entry pass
        beyond 2^23 entries with tight emission) + 3 scan kernels; emission; 3
        kernels per tile-id byte; ranges; render."""
        nt = self.ranges.shape[0]
        bits = 0
        while (1 << bits) < nt:
            bits += 1
        tile_passes = (bits + 7) // 8
        count = 0 if self.m > (1 << 23) else 1
        return 1 + 4 * 3 + (count + 3) + 1 + 3 * tile_passes + 1 + 1


def measure_peaks(dev, reps=5):
    """Throughput of the FP32 FMA pipe (scalar and packed two-wide FMA chains)
    and of the SFU's ex2 on this GPU, from the library's probe kernels (run
    outside the timed region), with the SM clock sampled during the probes."""
    import ctypes
    import torch
    from paper_2606_16566_gb300 import _lib as L
    lib = L.load()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(sms * 8, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {}
    with Clocks(dev.index) as clk:
        for name, kind, iters in (("ffma_tflops", L.PROBE_FFMA, 6000), ("ffma2_tflops", L.PROBE_FFMA2, 3000),
                                  ("ex2_tops", L.PROBE_EX2, 1500)):
            ts = []
            ops = ctypes.c_double(0)
            for _ in range(reps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                L.check(lib.lgs_peak_probe(kind, sms * 8, iters, ctypes.c_void_p(sink.data_ptr()),
                                           ctypes.byref(ops), stream), "lgs_peak_probe")
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            out[name] = ops.value / (statistics.median(ts[2:]) * 1e-3) / 1e12
    out["sm_mhz"] = clk.summary()["sm_mhz"]
    out["how"] = (f"lgs_peak_probe: {sms * 8} CTAs x 256 threads x 8 independent chains; median of {reps} "
                  "launches, CUDA events")
    return out


def loaded_clock_mhz():
    """Median SM clock of the GB300s under a power-capped sustained load,
    when the machine's measured-peaks record is present."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["clocks_under_load"]["sm_mhz_median"])
    except (OSError, KeyError, ValueError, TypeError):
        return None


def time_steps(pipe, cfg, steps, flush, backward=False):
    import torch
    ns = 4 if backward else 3
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(ns + 1)] for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        e = ev[i]
        e[0].record()
        pipe.stage_pre(cfg)
        e[1].record()
        pipe.stage_sort(cfg)
        e[2].record()
        pipe.stage_render(cfg)
        e[3].record()
        if backward:
            pipe.stage_backward(cfg)
            e[4].record()
    torch.cuda.synchronize()
    stage = np.array([[e[k].elapsed_time(e[k + 1]) for k in range(ns)] for e in ev])
    return stage  # [steps, stages] ms


def graph_steps(pipe, cfg, steps, flush, backward=False):
    """The same step (forward, or forward + backward) captured once in a CUDA
    graph and replayed `steps` times; L2 flushed before each replay, outside
    the events. Returns the per-replay times [steps] in ms."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        pipe.step(cfg)
        if backward:
            pipe.stage_backward(cfg)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        pipe.step(cfg)
        if backward:
            pipe.stage_backward(cfg)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        ev[i][0].record()
        graph.replay()
        ev[i][1].record()
    torch.cuda.synchronize()
    del graph
    return np.array([e[0].elapsed_time(e[1]) for e in ev])


def recorded_traffic(kernel="render_localgs_16x16"):
    """DRAM bytes per launch from the committed ncu record, or None once the
    kernel source no longer matches the profiled one."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = b"".join(open(os.path.join(ROOT, "paper_2606_16566_gb300", "csrc", f), "rb").read()
                       for f in ("render.cu", "common.cuh"))
        if hashlib.sha256(src).hexdigest()[:16] == rec["source_sha256_prefix"]:
            return rec["traffic_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        pass
    return None


def run_batched(dev, steps):
    """The batched workload: 3M clustered SH3 Gaussians, 64 cameras of uneven
    resolution; forward + backward captured in one CUDA graph with tight-box
    emission, tile shape and persistent launch picked by the autotuner, graph
    replays timed."""
    import torch
    from paper_2606_16566_gb300 import batch, lgs, scenes
    sc, cams = scenes.batched()
    g = lgs.to_device(sc, dev)
    del sc
    tune = batch.autotune(g, cams, backward=True, reps=3, use_cache=False, tight=True, batches=(256,))
    r = batch.Renderer(g, cams, tile=tune["tile"], persistent=tune["persistent"], backward=True, tight=True,
                       batch=tune["batch"], block=tune["block"])
    r.d_rgb.fill_(1.0 / r.d_rgb.numel())
    r.capture()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ts = []
    for i in range(max(3, steps // 4) + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r.graph.replay()
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            ts.append(e0.elapsed_time(e1))
    st = r.check()
    ms = float(np.median(ts))
    P = lgs.n_pixels(cams)
    out = {"workload": "batched-3M-sh3-64-uneven-views-fwd+bwd-graph", "emission": "tight",
           "view_groups": len(r.groups),
           "frames_s": len(cams) / (ms * 1e-3),
           "mpix_s": P / 1e6 / (ms * 1e-3), "ms_per_step": ms, "instances_K": int(st[2]),
           "tile": list(tune["tile"]), "warp_block": list(tune["block"]), "persistent": tune["persistent"],
           "staging_batch": tune["batch"],
           "autotune": tune["timings"],
           "replays": len(ts)}
    del r, g
    torch.cuda.empty_cache()
    return out, len(ts)


def _graph_ms(graph, flush, reps):
    import torch
    ts = []
    for i in range(reps + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        torch.cuda.synchronize()
        if i >= 2:
            ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), len(ts)


def run_indoor(dev, steps):
    """The indoor training step: 2.8M SH3 Gaussians on room walls, one 1332x876
    view; forward, L1 loss against a seeded random target, full adjoint, all in
    one CUDA graph (tight-box emission; tile shape, warp block and launch from
    the autotuner on forward + backward)."""
    import torch
    from paper_2606_16566_gb300 import batch, lgs, scenes
    sc, cams = scenes.indoor()
    g = lgs.to_device(sc, dev)
    del sc
    tune = batch.autotune(g, cams, backward=True, reps=3, use_cache=False, tight=True, batches=(256,))
    r = batch.Renderer(g, cams, tile=tune["tile"], persistent=tune["persistent"], backward=True, tight=True,
                       batch=tune["batch"], block=tune["block"])
    target = torch.rand(r.rgb.shape, generator=torch.Generator(device=dev).manual_seed(7), device=dev)
    diff = torch.empty_like(r.rgb)
    inv_n = 1.0 / r.rgb.numel()

    def step():
        r.forward()
        torch.sub(r.rgb, target, out=diff)
        torch.sign(diff, out=r.d_rgb)
        r.d_rgb.mul_(inv_n)
        r.backward()

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ms, n = _graph_ms(graph, flush, max(3, steps // 4))
    st = r.check()
    loss = float(diff.abs().mean().item())
    P = lgs.n_pixels(cams)
    out = {"workload": "indoor-2.8M-sh3-1332x876-training-step (fwd + L1 + bwd, graph, tight)",
           "steps_s": 1e3 / ms, "ms_per_step": ms, "mpix_s": P / 1e6 / (ms * 1e-3), "instances_K": int(st[2]),
           "l1_loss": loss, "replays": n, "tile": list(tune["tile"]), "warp_block": list(tune["block"]),
           "persistent": tune["persistent"], "autotune": tune["timings"]}
    del r, g, graph
    torch.cuda.empty_cache()
    return out


# tile shapes timed on the scale scene (8x8 warp blocks, batch 128): the
# larger tiles fit all 16 views in one view group of at most 2^16 tiles
SCALE_TILES = ((16, 16), (32, 16), (32, 32))


def _stage_times(r, flush, n):
    """Median per-stage (preprocess, sort, render) forward times of `n` eager
    steps after one warm-up, L2 flushed before each."""
    import torch
    stage = []
    for i in range(n + 1):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        r.stage_preprocess()
        e[1].record()
        r.stage_sort()
        e[2].record()
        r.stage_render()
        e[3].record()
        torch.cuda.synchronize()
        if i >= 1:
            stage.append([e[k].elapsed_time(e[k + 1]) for k in range(3)])
    return np.median(np.array(stage), 0)


def run_scale(dev, steps, tile=None, block=None):
    """The scale scene: 30M SH3 Gaussians (256 clusters + background), 16 views
    of 1920x1080 in one batch (view groups of at most 2^16 tiles); forward with
    per-stage events, forward+backward
    as one graph replay, the warp-culled fraction of the Local-GS schedule, and
    the HBM rate of preprocess (algorithmic bytes: 236 B read per Gaussian,
    69 B written per (view, Gaussian) entry). Without a fixed tile the forward
    of each shape in SCALE_TILES is timed and the fastest measured."""
    import torch
    from paper_2606_16566_gb300 import batch, lgs, scenes
    from paper_2606_16566_gb300 import _lib as L
    sc, cams = scenes.scale()
    g = lgs.to_device(sc, dev)
    del sc
    n, V = g["means"].shape[0], len(cams)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    tuned = None
    if tile is None:
        tuned = {}
        for t in SCALE_TILES:
            r = batch.Renderer(g, cams, tile=t, tight=True, block=(8, 8), batch=128)
            r.forward()
            tuned[f"{t[0]}x{t[1]}"] = float(_stage_times(r, flush, 2).sum())
            del r
            torch.cuda.empty_cache()
        best = min(tuned, key=tuned.get)
        tile, block, bsz = tuple(int(x) for x in best.split("x")), (8, 8), 128
    else:
        bsz = 0
    r = batch.Renderer(g, cams, tile=tile, backward=True, tight=True, block=block, batch=bsz)
    r.forward()
    pairs, cands = r.count_pairs()
    sm = _stage_times(r, flush, max(3, steps // 8))
    st = r.check()
    K = int(st[L.ST_NUM_INSTANCES])
    ms_f = float(sm.sum())
    r.d_rgb.fill_(1.0 / r.d_rgb.numel())
    r.capture()
    ms_fb, nrep = _graph_ms(r.graph, flush, max(3, steps // 8))
    r.check()
    P = lgs.n_pixels(cams)
    pre_bytes = n * 236 + n * V * 69
    out = {"workload": "scale-30M-sh3-16x1920x1080 (tight)", "tile": list(tile),
           "warp_block": list(block) if block else None, "staging_batch": bsz or 256,
           "tile_choice": {"forward_ms_by_tile": tuned} if tuned else "fixed",
           "frames_s": V / (ms_f * 1e-3),
           "mpix_s": P / 1e6 / (ms_f * 1e-3), "ms_per_step": ms_f,
           "stage_ms": {"preprocess": float(sm[0]), "sort": float(sm[1]), "render": float(sm[2])},
           "fwd_bwd": {"frames_s": V / (ms_fb * 1e-3), "ms_per_step": ms_fb, "replays": nrep},
           "view_groups": len(r.groups),
           "instances_K": K, "culled_warp_fraction": 1.0 - pairs / 32.0 / max(cands, 1),
           "warp_candidates": cands, "pairs": pairs,
           "preprocess_hbm_gbs": pre_bytes / (sm[0] * 1e-3) / 1e9,
           "preprocess_bytes": pre_bytes}
    del r, g
    torch.cuda.empty_cache()
    return out


def run_tiny(dev, steps):
    """The small configuration (10k Gaussians SH0, one 256x256 view, 16x16
    tiles, forward): every warp-block layout of the 16x16 tile timed as
    CUDA-graph replays of the whole step (eager sums beside), the fastest
    reported, and the oracle on full frames of the same view beside it."""
    import torch
    from paper_2606_16566_gb300 import lgs, scenes
    from paper_2606_16566_gb300 import _lib as L
    sc, cams = scenes.tiny()
    g = lgs.to_device(sc, dev)
    probe = lgs.render(g, cams, tile=(16, 16), flags=L.FLAG_TIGHT)
    pipe = Pipeline(g, cams, (16, 16), int(probe["K"] * 1.05) + 1024)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    per, eager = {}, {}
    for blk in lgs.WARP_BLOCKS[(16, 16)]:
        cfg = lgs.config((16, 16), "localgs", L.FLAG_TIGHT, 0, blk)
        for _ in range(3):
            pipe.step(cfg)
        name = f"{blk[0]}x{blk[1]}"
        eager[name] = float(np.median(time_steps(pipe, cfg, max(30, steps), flush).sum(1)))
        per[name] = float(np.median(graph_steps(pipe, cfg, max(30, steps), flush)))
    best = min(per, key=per.get)
    ms = per[best]
    out = {"workload": "tiny-10k-sh0-256x256 (16x16 tiles, tight, fwd)", "frames_s": 1e3 / ms,
           "mpix_s": 256 * 256 / 1e6 / (ms * 1e-3), "ms_per_step": ms, "timing": "graph replay",
           "block": best, "ms_by_block": per, "eager_ms_by_block": eager}
    out["cpu_baseline"] = cpu_baseline(sc, cams, budget_s=3.0, label="10k Gaussians")
    return out


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist
    from paper_2606_16566_gb300 import lgs, scenes
    from paper_2606_16566_gb300 import _lib as L

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    tile = (16, 16) if args.tile == "auto" else tuple(int(x) for x in args.tile.split("x"))
    block = None if args.block == "paper" else tuple(int(x) for x in args.block.split("x"))
    if args.profile and args.scene != "outdoor":
        from paper_2606_16566_gb300 import batch
        scene, cams = getattr(scenes, args.scene)()
        cams = cams[:args.views]
        g = lgs.to_device(scene, dev)
        del scene
        r = batch.Renderer(g, cams, tile=tile, mode=args.mode, backward=args.backward, tight=args.tight,
                           block=block, batch=args.batch)
        if args.backward:
            r.d_rgb.fill_(1.0 / r.d_rgb.numel())
        for _ in range(args.warmup + args.steps):
            r.forward()
            if args.backward:
                r.backward()
        torch.cuda.synchronize()
        r.check()
        return
    scene, cams = scenes.outdoor()
    cams = cams[:args.views]
    g = lgs.to_device(scene, dev)
    if args.profile:
        probe = lgs.render(g, cams, tile=tile)
        pipe = Pipeline(g, cams, tile, int(probe["K"] * 1.05) + 1024)
        del probe
        flags = (L.FLAG_TIGHT if args.tight else 0) | (L.FLAG_ONESWEEP if args.sort == "onesweep" else 0)
        cfg = lgs.config(tile, args.mode, flags, args.batch, block)
        if args.backward:
            pipe.setup_backward()
        for _ in range(args.warmup + args.steps):
            pipe.step(cfg)
            if args.backward:
                pipe.stage_backward(cfg)
        torch.cuda.synchronize()
        return
    TF = L.FLAG_TIGHT
    tuned = None
    persistent = 0
    nbat = args.batch
    if args.tile == "auto":
        # tile shape, warp-block layout, staging batch and launch of the
        # Local-GS forward from the project's autotuner (timed graph replays of
        # every candidate, outside the timed region)
        from paper_2606_16566_gb300 import batch
        tuned = batch.autotune(g, cams, tight=True, reps=5, use_cache=False)
        tile = tuple(tuned["tile"])
        block = tuple(tuned["block"])
        persistent = L.FLAG_PERSISTENT if tuned["persistent"] else 0
        nbat = tuned["batch"]
    paper_block = lgs.WARP_BLOCKS[tile][0]
    block = block or paper_block
    PF = persistent
    # the plain rasterizer runs on the standard 3DGS 16x16 tile, its own best
    # shape; the Local-GS variants on the tuned tile and block
    tile_p = (16, 16) if args.tile == "auto" else tile
    variants = {"localgs": lgs.config(tile, "localgs", PF, nbat, block), "plain": lgs.config(tile_p, "plain"),
                "localgs_tight": lgs.config(tile, "localgs", TF | PF, nbat, block),
                "plain_tight": lgs.config(tile_p, "plain", TF), "literal_tight": lgs.config(tile, "literal", TF)}
    if tuple(block) != tuple(paper_block):
        # the same tile in the paper's warp layout (eight full-width strips)
        variants["localgs_tight_paper_layout"] = lgs.config(tile, "localgs", TF, 0, paper_block)
    forward_only = {"literal_tight", "localgs_tight_paper_layout"}

    # discover K and size the instance buffers once per tile shape (outside the timed region)
    pipes_by_tile = {}
    for t in {tile, tile_p}:
        probe = lgs.render(g, cams, tile=t)
        pipes_by_tile[t] = Pipeline(g, cams, t, int(probe["K"] * 1.05) + 1024)
        del probe
    pipe = pipes_by_tile[tile]
    pipe_of = {name: pipes_by_tile[(cfg.tile_w, cfg.tile_h)] for name, cfg in variants.items()}
    # schedule work of the Local-GS render (pixel-Gaussian pairs) and K, counted once
    counts = {}
    for name, cfg in variants.items():
        q = pipe_of[name]
        q.step(lgs.with_flags(cfg, cfg.flags | L.FLAG_COUNT))
        st = lgs.read_status(q.status)
        if st[L.ST_CODE] != 0:
            raise L.LgsError(int(st[L.ST_CODE]), f"device status in {name}")
        counts[name] = {"pairs": int(st[L.ST_PAIRS]), "K": int(st[L.ST_NUM_INSTANCES])}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks = measure_peaks(dev)

    for q in pipes_by_tile.values():
        q.setup_backward()
    for _ in range(args.warmup):
        for name, cfg in variants.items():
            pipe_of[name].step(cfg)
            if name not in forward_only:
                pipe_of[name].stage_backward(cfg)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    n_bw = max(3, args.steps // 2)
    fwd, fb = {}, {}
    # the Local-GS / plain pair of the headline comparison is also timed as
    # CUDA-graph replays of the whole step (the way a renderer serves repeated
    # frames: one launch of the captured stages); the others eager only
    graphed = ("localgs_tight", "plain_tight")
    fwd_g, fb_g = {}, {}
    with Clocks(dev.index) as clk:
        for name, cfg in variants.items():
            fwd[name] = time_steps(pipe_of[name], cfg, args.steps, flush)
            if name not in forward_only:
                fb[name] = time_steps(pipe_of[name], cfg, n_bw, flush, backward=True)
        for name in graphed:
            fwd_g[name] = graph_steps(pipe_of[name], variants[name], args.steps, flush)
            fb_g[name] = graph_steps(pipe_of[name], variants[name], n_bw, flush, backward=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for q in pipes_by_tile.values():
        st = lgs.read_status(q.status)
        if st[L.ST_CODE] != 0:
            raise L.LgsError(int(st[L.ST_CODE]), "device status after the timed steps")
    # step time: the median of the timed steps (graph replays where timed so,
    # else each the sum of its eager stages)
    ms_eager = {n: float(np.median(fwd[n].sum(1))) for n in variants}
    ms_b_eager = {n: float(np.median(fb[n].sum(1))) for n in fb}
    ms = {n: float(np.median(fwd_g[n])) if n in fwd_g else ms_eager[n] for n in variants}
    ms_b = {n: float(np.median(fb_g[n])) if n in fb_g else ms_b_eager[n] for n in fb}
    names, names_b = list(ms), list(ms_b)
    vals = reduce_max_over_ranks([ms[n] for n in names] + [ms_b[n] for n in names_b], world, dev)
    ms = dict(zip(names, vals[:len(names)]))
    ms_b = dict(zip(names_b, vals[len(names):]))
    views = len(cams)
    P = lgs.n_pixels(cams)
    # headline: the faster of the two Local-GS emissions (both reported)
    head = min(("localgs", "localgs_tight"), key=lambda n: ms_eager[n])
    ms_l = ms[head]
    fps = world * views / (ms_l * 1e-3)
    stage_ms = np.median(fwd[head], 0)
    # the render kernel's average launch time over the timed steps (CUDA events
    # around its one launch per step, on the launching stream)
    render_ms = float(fwd[head][:, 2].mean())
    pairs = counts[head]["pairs"]
    achieved = pairs * 19.0 / (render_ms * 1e-3) / 1e12
    peak = max(peaks["ffma_tflops"], peaks["ffma2_tflops"])
    sfu_rate = pairs / (render_ms * 1e-3) / 1e12
    cfg_l = variants[head]
    loaded = loaded_clock_mhz()
    probe_mhz = peaks["sm_mhz"] or 2070.0
    # issue roofline: the 16 per-pixel operations the definition needs per
    # pair (5 FMA power, ex2, clamp, 1/255 test, T(1 - alpha), stop test, w,
    # 3 FMA colour, T update, contributor index) against 32 lanes x one warp
    # instruction per scheduler per clock (4 schedulers per SM) at the probe clock
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = n_sm * 4 * 32 * probe_mhz * 1e6 / 1e12
    issue = {"ops_per_pair": 16, "achieved": pairs * 16.0 / (render_ms * 1e-3) / 1e12, "peak": issue_peak,
             "unit": "T lane-ops/s", "frac": pairs * 16.0 / (render_ms * 1e-3) / 1e12 / issue_peak,
             "peak_basis": f"{n_sm} SMs x 4 schedulers x 32 lanes x {probe_mhz:.0f} MHz"}

    def summary(name):
        f = np.median(fwd[name], 0)
        out = {"frames_s": world * views / (ms[name] * 1e-3), "mpix_s": world * P / 1e6 / (ms[name] * 1e-3),
               "ms_per_step": ms[name], "timing": "graph replay" if name in fwd_g else "eager",
               "eager_ms_per_step": ms_eager[name],
               "stage_ms": {"preprocess": float(f[0]), "sort": float(f[1]), "render": float(f[2])},
               "instances_K": counts[name]["K"], "pairs": counts[name]["pairs"]}
        if name in fb:
            b = np.median(fb[name], 0)
            out["fwd_bwd"] = {"frames_s": world * views / (ms_b[name] * 1e-3),
                              "mpix_s": world * P / 1e6 / (ms_b[name] * 1e-3), "ms_per_step": ms_b[name],
                              "eager_ms_per_step": ms_b_eager[name], "backward_ms": float(b[3])}
        return out

    # end to end: host scene -> device, pipeline, image -> host, every step.
    # Two buffer sets and three streams pipeline consecutive steps: step i's
    # upload, step i-1's render and step i-2's download overlap, as a serving
    # loop would run them; every step still moves its full inputs and image.
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).pin_memory() for k in g}
        out_h = [torch.empty(pipe.rgb.numel(), dtype=torch.float32).pin_memory() for _ in range(2)]
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = out_h[0].numel() * 4
        gs = [g, {k: torch.empty_like(v) for k, v in g.items()}]
        pipes = [pipe, Pipeline(gs[1], cams, tile, pipe.capacity)]
        # each buffer set's step captured once as a CUDA graph (as the device
        # timing of the headline), replayed on the compute stream
        graphs = []
        for q in pipes:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                q.step(cfg_l)
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr):
                q.step(cfg_l)
            graphs.append(gr)
        s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_cmp = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        torch.cuda.synchronize()
        for e in ev_in + ev_cmp + ev_out:
            e.record()

        def e2e_step(i):
            b = i & 1
            with torch.cuda.stream(s_in):
                s_in.wait_event(ev_cmp[b])            # scene buffer b is free again
                for k in gs[b]:
                    gs[b][k].copy_(host[k], non_blocking=True)
                ev_in[b].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[b])
                s_cmp.wait_event(ev_out[b])           # image buffer b was read back
                graphs[b].replay()
                ev_cmp[b].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_cmp[b])
                out_h[b].copy_(pipes[b].rgb, non_blocking=True)
                ev_out[b].record(s_out)

        for i in range(4):
            e2e_step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_e2e = max(6, args.steps // 2)
        e0.record(s_in)
        for i in range(n_e2e):
            e2e_step(i)
        s_in.wait_stream(s_out)
        e1.record(s_in)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1) / n_e2e
        for q in pipes:
            st = lgs.read_status(q.status)
            if st[L.ST_CODE] != 0:
                raise L.LgsError(int(st[L.ST_CODE]), "device status in the end-to-end steps")
        ms_e2e = reduce_max_over_ranks([ms_e2e], world, dev)[0]
        # the copies alone (same tensors, same streams, nothing overlapping):
        # the end-to-end step is bound by max(device step, upload, download)
        copy_ms = {}
        for name, fn, strm in (("h2d", lambda: [gs[0][k].copy_(host[k], non_blocking=True) for k in gs[0]], s_in),
                               ("d2h", lambda: out_h[0].copy_(pipes[0].rgb, non_blocking=True), s_out)):
            with torch.cuda.stream(strm):
                fn()
                c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                c0.record(strm)
                for _ in range(5):
                    fn()
                c1.record(strm)
            torch.cuda.synchronize()
            copy_ms[name] = c0.elapsed_time(c1) / 5
        e2e = {"value": world * views / (ms_e2e * 1e-3), "unit": "frames/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
               "copy_alone_ms": copy_ms,
               "copy_alone_gbs": {"h2d": h2d / (copy_ms["h2d"] * 1e6), "d2h": d2h / (copy_ms["d2h"] * 1e6)},
               "schedule": "2 buffer sets, upload / render (one CUDA-graph replay of the whole step) / download "
                           "of consecutive steps on 3 streams"}
        del graphs, pipes[1], gs[1]

    tiny = None if args.no_tiny else run_tiny(dev, args.steps)
    batched, n_batched = (None, 0)
    if not args.no_batched:
        batched, n_batched = run_batched(dev, args.steps)
    indoor = None if args.no_indoor else run_indoor(dev, args.steps)
    scale = None if args.no_scale else (run_scale(dev, args.steps) if args.tile == "auto"
                                        else run_scale(dev, args.steps, tile, block))
    if rank != 0:
        return
    emission = "tight" if head.endswith("tight") else "rect"
    plain_same = "plain_tight" if emission == "tight" else "plain"
    s_head, s_plain = summary(head), summary(plain_same)
    line = {
        "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "views_per_step": views, "gaussians": pipe.n,
                   "tile": f"{tile[0]}x{tile[1]}", "warp_block": f"{block[0]}x{block[1]}",
                   "persistent": bool(persistent), "staging_batch": nbat or 256,
                   "tile_choice": "autotuned" if tuned else "fixed",
                   "plain_tile": f"{tile_p[0]}x{tile_p[1]}",
                   "emission": emission, "instances_K": counts[head]["K"],
                   "step_time": f"median of {args.steps} timed steps: CUDA-graph replays of the whole step "
                                f"for the Local-GS and plain tight-emission variants (their stage times from eager "
                                f"per-stage events), eager stage sums for the other variants",
                   "l2": "flushed between steps (256 MB write, outside the events)",
                   "parallelism": f"replicas x{world}"},
        "variants": {n: summary(n) for n in variants},
        "upstream_grad": "fixed +-1/numel dL/drgb (L1-loss shaped), 3D grads zeroed each step",
        "autotune": tuned["timings"] if tuned else None,
        "peaks": peaks,
        "batched": batched,
        "indoor": indoor,
        "scale": scale,
        "tiny": tiny,
        "gpu_launches": sum(pipe_of[n].launches() * args.steps for n in variants)
                        + sum((pipe_of[n].launches() + 2) * n_bw for n in fb)
                        + sum(pipe_of[n].launches() * args.steps + (pipe_of[n].launches() + 2) * n_bw
                              for n in fwd_g),
        "clocks": clk.summary(),
        "e2e": e2e,
        "roofline": {"bound": "alu", "kernel": "render_localgs" + ("_persistent" if persistent else ""),
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": recorded_traffic(f"render_localgs{'_persistent' if persistent else ''}"
                                                 f"_{tile[0]}x{tile[1]}_{block[0]}x{block[1]}_{emission}"),
                     "work": f"{pairs} pixel-Gaussian pairs x 19 FP32 flops",
                     "peak_basis": f"measured: FP32 FMA-chain probe (scalar {peaks['ffma_tflops']:.1f}, "
                                   f"packed {peaks['ffma2_tflops']:.1f} TFLOP/s) at {probe_mhz:.0f} MHz",
                     "peak_at_loaded_clock": peak * loaded / probe_mhz if loaded else None,
                     "loaded_clock_mhz": loaded,
                     "sfu": {"achieved": sfu_rate, "peak": peaks["ex2_tops"], "unit": "T ex2/s",
                             "frac": sfu_rate / peaks["ex2_tops"]},
                     "issue": issue},
        "comparison": {
            "localgs_fwd_frames_s": fps, "plain_fwd_frames_s": s_plain["frames_s"],
            "fwd_ratio": s_plain["ms_per_step"] / ms_l,
            "localgs_fwd_bwd_frames_s": s_head["fwd_bwd"]["frames_s"],
            "plain_fwd_bwd_frames_s": s_plain["fwd_bwd"]["frames_s"],
            "fwd_bwd_ratio": s_plain["fwd_bwd"]["ms_per_step"] / s_head["fwd_bwd"]["ms_per_step"],
            "render_kernel_ratio": float(np.median(fwd[plain_same][:, 2])) / float(np.median(fwd[head][:, 2])),
            "localgs_mpix_s": s_head["mpix_s"], "plain_mpix_s": s_plain["mpix_s"],
            "stage_ms": s_head["stage_ms"], "backward_ms": s_head["fwd_bwd"]["backward_ms"],
            "emission": emission, "tile": f"{tile[0]}x{tile[1]}", "warp_block": f"{block[0]}x{block[1]}",
            "plain_tile": f"{tile_p[0]}x{tile_p[1]}",
            "batched_fwd_bwd_frames_s": batched["frames_s"] if batched else None,
            "indoor_steps_s": indoor["steps_s"] if indoor else None,
            "scale_fwd_frames_s": scale["frames_s"] if scale else None,
            "scale_fwd_bwd_frames_s": scale["fwd_bwd"]["frames_s"] if scale else None,
            "tiny_fwd_frames_s": tiny["frames_s"] if tiny else None},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cams)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
