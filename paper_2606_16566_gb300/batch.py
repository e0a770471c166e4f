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

``autotune`` times the candidate tile shapes (16x16, 8x32, 32x8) with every
warp-block layout of the Local-GS render for that shape (the paper's
full-width strips, 2D blocks, two-pixels-per-lane blocks) and staging batches
of 256 or 128 Gaussians, then the persistent launch of the best of them, on
the actual workload, and caches the fastest per (Gaussian-count bucket,
pixel-count bucket, view count, mode, emission).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import _lib as L
from . import lgs

TILE_SHAPES = ((16, 16), (8, 32), (32, 8), (32, 32), (16, 32), (32, 16))
# tiles of 256 pixels: the only ones of the plain and study kernels
SMALL_TILE_SHAPES = ((16, 16), (8, 32), (32, 8))


MAX_GROUP_TILES = 1 << 16


def view_groups(cams, tile, max_tiles=MAX_GROUP_TILES):
    """Consecutive view groups [(v0, v1)] with at most max_tiles tiles (and at
    most LGS_MAX_VIEWS views) each: inside a group tile ids fit in 16 bits, so
    its tile-id sort takes two radix passes instead of three."""
    tw, th = tile
    groups, v0, acc = [], 0, 0
    for v, c in enumerate(cams):
        t = ((c["width"] + tw - 1) // tw) * ((c["height"] + th - 1) // th)
        if v > v0 and (acc + t > max_tiles or v - v0 >= L.LGS_MAX_VIEWS):
            groups.append((v0, v))
            v0, acc = v, 0
        acc += t
    groups.append((v0, len(cams)))
    return groups


class Renderer:
    """All buffers of the pipeline for a fixed camera set, eager or as one
    CUDA graph. Views are processed in groups of at most MAX_GROUP_TILES tiles
    (one group for most batches): one preprocess call for all views, then a
    sort, render and adjoint call per group on that group's rows of the
    preprocess outputs, pixels and 2D gradients (so a group's lists hold
    indices into its own rows; lists() gives the global form). A tile's list
    depends only on the entries of its own view, so grouping changes no
    output."""

    def __init__(self, g, cams, tile=(16, 16), mode="localgs", persistent=False, capacity=None,
                 headroom=1.10, backward=False, tight=False, max_group_tiles=MAX_GROUP_TILES, batch=0,
                 block=None):
        self.g, self.cams, self.tile, self.mode = g, cams, tuple(tile), mode
        flags = (L.FLAG_PERSISTENT if persistent else 0) | (L.FLAG_TIGHT if tight else 0)
        self.cfg = lgs.config(tile, mode, flags, batch, block)
        self.carr = lgs.cameras(cams)
        dev = g["means"].device
        self.n = g["means"].shape[0]
        self.m = max(self.n * len(cams), 1)
        self.groups = view_groups(cams, self.tile, max_group_tiles)
        if capacity is None:
            caps = []
            for v0, v1 in self.groups:
                probe = lgs.render(g, cams[v0:v1], tile=tile, mode=mode, flags=L.FLAG_TIGHT if tight else 0)
                caps.append(int(math.ceil(probe["K"] * headroom)) + 1024)
                del probe
        else:
            caps = [int(capacity)] * len(self.groups) if len(self.groups) == 1 else list(capacity)
        self.capacity = sum(caps)
        self.pre = lgs.PreOut.empty(self.m, dev)
        self.vals = torch.empty(self.capacity, dtype=torch.int32, device=dev)
        self.ranges = torch.empty((lgs.n_tiles(cams, self.cfg), 2), dtype=torch.int32, device=dev)
        self.ws = torch.empty(max(lgs.sort_workspace_size(self.n * (v1 - v0), c)
                                  for (v0, v1), c in zip(self.groups, caps)), dtype=torch.uint8, device=dev)
        P = lgs.n_pixels(cams)
        self.rgb = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.T = torch.empty(P, dtype=torch.float32, device=dev)
        self.nc = torch.empty(P, dtype=torch.int32, device=dev)
        self.backward_enabled = backward
        if backward:
            self.d_rgb = torch.zeros(3 * P, dtype=torch.float32, device=dev)
            self.d_T = None
            self.grads = lgs.new_grads(g, len(cams))
        # per-group views of the buffers
        self.parts = []
        voff = toff = poff = 0
        for (v0, v1), cap in zip(self.groups, caps):
            cg = cams[v0:v1]
            nt, npx = lgs.n_tiles(cg, self.cfg), lgs.n_pixels(cg)
            part = {"cams": cg, "carr": lgs.cameras(cg), "cap": cap, "voff": voff, "toff": toff,
                    "pre": self.pre.rows(v0 * self.n, v1 * self.n), "vals": self.vals[voff:voff + cap],
                    "ranges": self.ranges[toff:toff + nt], "rgb": self.rgb[3 * poff:3 * (poff + npx)],
                    "T": self.T[poff:poff + npx], "nc": self.nc[poff:poff + npx],
                    "status": lgs.new_status(dev)}
            if backward:
                part["d_rgb"] = self.d_rgb[3 * poff:3 * (poff + npx)]
                part["grads"] = dict(self.grads)
                for k, w in (("xy2d", 2), ("conic2d", 4), ("rgb2d", 4)):
                    part["grads"][k] = self.grads[k][v0 * self.n:v1 * self.n]
            self.parts.append(part)
            voff, toff, poff = voff + cap, toff + nt, poff + npx
        self.status = self.parts[0]["status"]
        self.graph = None

    # ------------------------------------------------------------------ eager
    def stage_preprocess(self, stream=None):
        for q in self.parts:
            q["status"].zero_()
        lgs.preprocess(self.g, self.carr, self.cfg, out=self.pre, status=self.status, stream=stream)

    def stage_sort(self, stream=None):
        for q in self.parts:
            lgs.sort(q["pre"], self.n, q["cams"], self.cfg, q["cap"], None, q["vals"], q["ranges"],
                     self.ws, q["status"], stream=stream, with_keys=False)

    def stage_render(self, cfg=None, stream=None):
        for q in self.parts:
            lgs.render_fwd(q["pre"], q["vals"], q["ranges"], q["cams"], cfg or self.cfg, q["rgb"], q["T"],
                           q["nc"], q["status"], stream=stream)

    def forward(self, stream=None):
        self.stage_preprocess(stream)
        self.stage_sort(stream)
        self.stage_render(stream=stream)

    def count_pairs(self):
        """(pixel-Gaussian pairs, warp candidates) of the Local-GS schedule over
        all groups (an extra render with LGS_FLAG_COUNT after a forward)."""
        cfg = lgs.with_flags(self.cfg, self.cfg.flags | L.FLAG_COUNT)
        for q in self.parts:
            q["status"][L.ST_PAIRS] = 0
            q["status"][L.ST_CANDIDATES] = 0
        self.stage_render(cfg)
        st = self.check()
        return int(st[L.ST_PAIRS]), int(st[L.ST_CANDIDATES])

    def backward(self, stream=None):
        for k in ("means", "scales", "quats", "opacities", "sh"):
            self.grads[k].zero_()
        for q in self.parts:
            lgs.render_bwd(self.g, q["cams"], self.cfg, q["pre"], q["vals"], q["ranges"], q["T"], q["nc"],
                           q["d_rgb"], self.d_T, q["grads"], q["status"], stream=stream)

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
        """Reads the device status of every group; raises on a device-side
        error. Returns the status words with the instance counts summed."""
        total = None
        for q in self.parts:
            st = lgs.read_status(q["status"])
            if st[L.ST_CODE] != 0:
                raise L.LgsError(int(st[L.ST_CODE]), f"device status (detail {int(st[L.ST_DETAIL])})")
            if total is None:
                total = st.copy()
            else:
                for w in (L.ST_NUM_INSTANCES, L.ST_NONFINITE, L.ST_PAIRS, L.ST_CANDIDATES):
                    total[w] += st[w]
        return total

    def lists(self):
        """(vals, ranges) of all groups as one list set: ranges index vals and
        vals are entry indices v*N + i over all views (a group's own lists hold
        indices into its own rows of the preprocess outputs)."""
        ranges = self.ranges.clone()
        vals = self.vals.clone()
        for (v0, _), q in zip(self.groups, self.parts):
            r = ranges[q["toff"]:q["toff"] + q["ranges"].shape[0]]
            nonempty = r[:, 1] > r[:, 0]
            r[nonempty] += q["voff"]
            vals[q["voff"]:q["voff"] + q["cap"]] += v0 * self.n
        return vals, ranges

    def images(self):
        return lgs.split_views(self.rgb, self.cams, 3)


def _bucket_key(n, cams, mode, backward, tight=False):
    P = lgs.n_pixels(cams)
    return (f"N2^{int(round(math.log2(max(n, 1))))}|P2^{int(round(math.log2(max(P, 1))))}|V{len(cams)}|"
            f"{mode}|{'fb' if backward else 'f'}{'|tight' if tight else ''}")


def default_cache_path():
    return os.path.join(os.path.expanduser("~"), ".cache", "lgs_autotune.json")


def autotune(g, cams, mode="localgs", backward=False, shapes=TILE_SHAPES, persistent=(False, True),
             reps=10, cache_path=None, use_cache=True, tight=False, batches=(256, 128), blocks=True):
    """Times every (tile shape, warp block, staging batch) candidate with graph
    replays, then the persistent launch of the fastest, and returns {"tile":
    (w, h), "block": (bw, bh), "persistent": bool, "batch": b, "ms": t,
    "timings": [...]}. blocks=False keeps the paper's full-width strips."""
    cache_path = cache_path or default_cache_path()
    key = _bucket_key(g["means"].shape[0], cams, mode, backward, tight)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
        if key in cache and "block" in cache[key]:
            c = cache[key]
            return {"tile": tuple(c["tile"]), "block": tuple(c["block"]), "persistent": c["persistent"],
                    "batch": c.get("batch", 256), "ms": c["ms"], "timings": c.get("timings", []),
                    "cached": True}
    timings = []
    caps = {}

    def run(tile, block, pers, nb):
        r = Renderer(g, cams, tile=tile, mode=mode, persistent=pers, backward=backward, tight=tight,
                     batch=nb, block=block, capacity=caps.get(tuple(tile)))
        caps.setdefault(tuple(tile), [p["cap"] for p in r.parts] if len(r.parts) > 1 else r.parts[0]["cap"])
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
        timings.append({"tile": list(tile), "block": list(block), "persistent": pers, "batch": nb,
                        "ms": float(np.median(ts[2:]))})
        del r
        torch.cuda.empty_cache()

    for tile in shapes:
        if mode != "localgs" and tuple(tile) not in SMALL_TILE_SHAPES:
            continue
        layouts = lgs.WARP_BLOCKS[tuple(tile)] if (blocks and mode == "localgs") else \
            lgs.WARP_BLOCKS[tuple(tile)][:1]
        for block in layouts:
            for nb in (batches if mode == "localgs" else (256,)):
                run(tile, block, False, nb)
    if mode == "localgs" and True in persistent:
        best = min(timings, key=lambda t: t["ms"])
        run(tuple(best["tile"]), tuple(best["block"]), True, best["batch"])
    best = min(timings, key=lambda t: t["ms"])
    cache[key] = {"tile": best["tile"], "block": best["block"], "persistent": best["persistent"],
                  "batch": best["batch"], "ms": best["ms"], "timings": timings}
    try:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    except OSError:
        pass
    return {"tile": tuple(best["tile"]), "block": tuple(best["block"]), "persistent": best["persistent"],
            "batch": best["batch"], "ms": best["ms"], "timings": timings, "cached": False}
