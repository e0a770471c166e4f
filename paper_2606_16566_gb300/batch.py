"""Batched multi-view rendering: preallocated buffers, CUDA-graph capture and
an autotuner.

``Renderer`` holds every buffer of the pipeline for a fixed set of cameras
(the library allocates nothing, so all of them are torch tensors), runs the
forward (and optionally the backward) through the C ABI, and can capture the
whole sequence -- status reset, preprocess, sort, render, gradient reset and
adjoint -- in one CUDA graph that later replays with a single launch call.
Cameras and the instance capacity are baked into a captured graph; scene
tensors and the upstream gradient are read in place, so they may change
between replays.

``autotune`` times the candidate tile shapes (16x16, 8x32, 32x8: the warp
strip of a 256-thread tile is 16x2, 8x4 or 32x1 pixels) with and without the
persistent render launch on the actual workload and caches the fastest per
(Gaussian-count bucket, pixel-count bucket, view count, mode).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import _lib as L
from . import lgs

TILE_SHAPES = ((16, 16), (8, 32), (32, 8))


class Renderer:
    def __init__(self, g, cams, tile=(16, 16), mode="localgs", persistent=False, capacity=None,
                 headroom=1.10, backward=False, tight=False):
        self.g, self.cams, self.tile, self.mode = g, cams, tuple(tile), mode
        flags = (L.FLAG_PERSISTENT if persistent else 0) | (L.FLAG_TIGHT if tight else 0)
        self.cfg = lgs.config(tile, mode, flags)
        self.carr = lgs.cameras(cams)
        dev = g["means"].device
        self.n = g["means"].shape[0]
        self.m = max(self.n * len(cams), 1)
        if capacity is None:
            probe = lgs.render(g, cams, tile=tile, mode=mode, flags=L.FLAG_TIGHT if tight else 0)
            capacity = int(math.ceil(probe["K"] * headroom)) + 1024
            del probe
        self.capacity = capacity
        self.status = lgs.new_status(dev)
        self.pre = lgs.PreOut.empty(self.m, dev)
        self.vals = torch.empty(capacity, dtype=torch.int32, device=dev)
        self.ranges = torch.empty((lgs.n_tiles(cams, self.cfg), 2), dtype=torch.int32, device=dev)
        self.ws = torch.empty(lgs.sort_workspace_size(self.n * len(cams), capacity), dtype=torch.uint8,
                              device=dev)
        P = lgs.n_pixels(cams)
        self.rgb = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.T = torch.empty(P, dtype=torch.float32, device=dev)
        self.nc = torch.empty(P, dtype=torch.int32, device=dev)
        self.backward_enabled = backward
        if backward:
            self.d_rgb = torch.zeros(3 * P, dtype=torch.float32, device=dev)
            self.d_T = None
            self.grads = lgs.new_grads(g, len(cams))
        self.graph = None

    # ------------------------------------------------------------------ eager
    def forward(self, stream=None):
        self.status.zero_()
        lgs.preprocess(self.g, self.carr, self.cfg, out=self.pre, status=self.status, stream=stream)
        lgs.sort(self.pre, self.n, self.cams, self.cfg, self.capacity, None, self.vals, self.ranges,
                 self.ws, self.status, stream=stream, with_keys=False)
        lgs.render_fwd(self.pre, self.vals, self.ranges, self.cams, self.cfg, self.rgb, self.T, self.nc,
                       self.status, stream=stream)

    def backward(self, stream=None):
        for k in ("means", "scales", "quats", "opacities", "sh"):
            self.grads[k].zero_()
        lgs.render_bwd(self.g, self.cams, self.cfg, self.pre, self.vals, self.ranges, self.T, self.nc,
                       self.d_rgb, self.d_T, self.grads, self.status, stream=stream)

    def step(self):
        if self.graph is not None:
            self.graph.replay()
            return
        self.forward()
        if self.backward_enabled:
            self.backward()

    # ------------------------------------------------------------------ graph
    def capture(self, warmup=2):
        """Captures forward (+ backward if enabled) in one CUDA graph."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.forward()
                if self.backward_enabled:
                    self.backward()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.forward()
            if self.backward_enabled:
                self.backward()
        return self

    def check(self):
        """Reads the device status; raises on a device-side error."""
        st = lgs.read_status(self.status)
        if st[L.ST_CODE] != 0:
            raise L.LgsError(int(st[L.ST_CODE]), f"device status (detail {int(st[L.ST_DETAIL])})")
        return st

    def images(self):
        return lgs.split_views(self.rgb, self.cams, 3)


def _bucket_key(n, cams, mode, backward, tight=False):
    P = lgs.n_pixels(cams)
    return (f"N2^{int(round(math.log2(max(n, 1))))}|P2^{int(round(math.log2(max(P, 1))))}|V{len(cams)}|"
            f"{mode}|{'fb' if backward else 'f'}{'|tight' if tight else ''}")


def default_cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "lgs_autotune.json")


def autotune(g, cams, mode="localgs", backward=False, shapes=TILE_SHAPES, persistent=(False, True),
             reps=10, cache_path=None, use_cache=True, tight=False):
    """Times every (tile shape, persistent) candidate with graph replays and
    returns {"tile": (w, h), "persistent": bool, "ms": t, "timings": [...]}."""
    cache_path = cache_path or default_cache_path()
    key = _bucket_key(g["means"].shape[0], cams, mode, backward, tight)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            c = cache[key]
            return {"tile": tuple(c["tile"]), "persistent": c["persistent"], "ms": c["ms"],
                    "timings": c.get("timings", []), "cached": True}
    timings = []
    for tile in shapes:
        for pers in persistent:
            if pers and mode != "localgs":
                continue
            r = Renderer(g, cams, tile=tile, mode=mode, persistent=pers, backward=backward, tight=tight)
            if backward:
                r.d_rgb.fill_(1.0 / r.d_rgb.numel())
            r.capture()
            ts = []
            for _ in range(reps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r.graph.replay()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            r.check()
            timings.append({"tile": list(tile), "persistent": pers, "ms": float(np.median(ts[2:]))})
            del r
            torch.cuda.empty_cache()
    best = min(timings, key=lambda t: t["ms"])
    cache[key] = {"tile": best["tile"], "persistent": best["persistent"], "ms": best["ms"],
                  "timings": timings}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    except OSError:
        pass
    return {"tile": tuple(best["tile"]), "persistent": best["persistent"], "ms": best["ms"],
            "timings": timings, "cached": False}
