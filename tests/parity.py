"""Comparison helpers for GPU-vs-oracle parity tests.

Tolerances (image: max |error| <= 2e-3 per channel and at most 1e-4 of the
pixels above 1e-5; integer outputs bit-exact outside the guard bands) are the
parity bar of the hot path. Guard items are decisions whose FP64 margin lies
inside the guard band of the oracle (oracle.DEFAULT_GUARD); they are counted
and must stay below 1e-4 of the items.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle

IMG_MAX_ABS = 2e-3
IMG_FINE = 1e-5
IMG_FINE_FRAC = 1e-4
GUARD_FRAC = 1e-4


def gpu_pre_numpy(pre, m):
    xy = pre.xy[:m].double().cpu().numpy()
    return {
        "uv": np.stack([xy[:, 0] + xy[:, 2], xy[:, 1] + xy[:, 3]], 1),
        "conic": pre.conic[:m, :3].double().cpu().numpy(),
        "opacity": pre.conic[:m, 3].cpu().numpy(),
        "rgb": pre.rgb[:m, :3].double().cpu().numpy(),
        "depth_bits": pre.depth[:m].cpu().numpy().view(np.uint32),
        "radius": pre.radius[:m].cpu().numpy(),
        "tiles": pre.tiles[:m].cpu().numpy().view(np.uint32).astype(np.int64),
        "rect": unpack_rect(pre.rect[:m].cpu().numpy().view(np.uint64)),
        "flags": pre.flags[:m].cpu().numpy(),
    }


def unpack_rect(r):
    r = r.astype(np.uint64)
    return np.stack([(r & 0xFFFF), (r >> 16) & 0xFFFF, (r >> 32) & 0xFFFF, (r >> 48) & 0xFFFF],
                    1).astype(np.int32)


def tile_lists(vals, ranges):
    out = []
    for s, e in ranges:
        out.append(vals[s:e])
    return out


def compare_preprocess(g, o, guard_mask):
    """Integer fields bit-exact outside guard Gaussians; returns a report dict."""
    ok = ~guard_mask
    rep = {}
    rep["radius_mismatch"] = int(np.sum((g["radius"] != o["radius"]) & ok))
    rep["tiles_mismatch"] = int(np.sum((g["tiles"] != o["tiles"]) & ok))
    vis = (o["tiles"] > 0) & (g["tiles"] > 0)
    rep["rect_mismatch"] = int(np.sum(np.any(g["rect"] != o["rect"], 1) & vis & ok))
    rep["depth_mismatch"] = int(np.sum((g["depth_bits"] != o["depth_bits"]) & ok))
    rep["guard"] = int(guard_mask.sum())
    if vis.any():
        rep["uv_max_err"] = float(np.max(np.abs(g["uv"][vis] - o["uv"][vis])))
        rel = np.abs(g["conic"][vis] - o["conic"][vis]) / (np.abs(o["conic"][vis]).max(1, keepdims=True))
        rep["conic_max_rel"] = float(rel.max())
        rep["rgb_max_err"] = float(np.max(np.abs(g["rgb"][vis] - o["rgb"][vis])))
    return rep


def guard_gaussians(o_pre):
    return o_pre["gflags"] != 0


def list_mismatch_tiles(g_vals, g_ranges, o_vals, o_ranges):
    bad = []
    for t in range(len(o_ranges)):
        gs, ge = g_ranges[t]
        os_, oe = o_ranges[t]
        if ge - gs != oe - os_ or not np.array_equal(g_vals[gs:ge], o_vals[os_:oe]):
            bad.append(t)
    return np.array(bad, dtype=np.int64)


def explained_by_guards(bad_tiles, o_vals, o_ranges, g_vals, g_ranges, guard_ids):
    """A differing tile list is explained when the symmetric difference of the
    two lists (as multisets of ids, plus order swaps) involves only guard
    Gaussians."""
    gset = set(int(i) for i in guard_ids)
    unexplained = []
    for t in bad_tiles:
        a = list(o_vals[o_ranges[t][0]:o_ranges[t][1]])
        b = list(g_vals[g_ranges[t][0]:g_ranges[t][1]])
        a2 = [x for x in a if int(x) not in gset]
        b2 = [x for x in b if int(x) not in gset]
        if a2 != b2:
            unexplained.append(int(t))
    return unexplained


def tile_pixel_mask(tiles, W, H, tw, th):
    gx = (W + tw - 1) // tw
    m = np.zeros((H, W), bool)
    for t in tiles:
        ty, tx = divmod(int(t), gx)
        m[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw] = True
    return m


def image_report(img_g, img_o, exclude):
    """img_*: [3,H,W]. exclude: [H,W] guard pixels."""
    err = np.abs(img_g.astype(np.float64) - img_o)
    perpix = err.max(0)
    keep = ~exclude
    return {
        "max_abs": float(perpix[keep].max()) if keep.any() else 0.0,
        "max_abs_all": float(perpix.max()),
        "frac_above_fine": float(np.mean(perpix[keep] > IMG_FINE)) if keep.any() else 0.0,
        "n_excluded": int(exclude.sum()),
        "n_pix": int(perpix.size),
    }


def assert_image_parity(rep, what=""):
    assert rep["max_abs"] <= IMG_MAX_ABS, (what, rep)
    assert rep["frac_above_fine"] <= IMG_FINE_FRAC, (what, rep)
    assert rep["n_excluded"] <= max(1, GUARD_FRAC * rep["n_pix"]) or rep["n_excluded"] <= 64, (what, rep)


def full_view_parity(scene, cam, res_gpu_view, tile, oracle_res=None):
    """Compares one view of a GPU render (dict from lgs.render split per view,
    already on the host as numpy) with the oracle. Returns reports."""
    tw, th = tile
    o = oracle_res if oracle_res is not None else oracle.render(scene, cam, tw, th)
    W, H = cam["width"], cam["height"]
    g_vals, g_ranges = res_gpu_view["vals"], res_gpu_view["ranges"]
    bad = list_mismatch_tiles(g_vals, g_ranges, o["vals"], o["ranges"])
    guard_ids = np.nonzero(guard_gaussians(o["pre"]))[0]
    unexplained = explained_by_guards(bad, o["vals"], o["ranges"], g_vals, g_ranges, guard_ids)
    excl = tile_pixel_mask(bad, W, H, tw, th) | (o["pguard"] != 0)
    rep = image_report(res_gpu_view["rgb"], o["rgb"], excl)
    nc_ok = (res_gpu_view["n_contrib"] == o["n_contrib"]) | excl
    rep["n_contrib_mismatch"] = int((~nc_ok).sum())
    rep["T_max_abs"] = float(np.max(np.abs(res_gpu_view["final_T"] - o["final_T"])[~excl])) if (~excl).any() else 0.0
    rep["bad_tiles"] = len(bad)
    rep["unexplained_tiles"] = unexplained
    return rep, o


def to_numpy_view(res, v, cams, n, tile):
    """Per-view host copies of a batched GPU render (vals re-based to the view)."""
    tw, th = tile
    cam = cams[v]
    gx = (cam["width"] + tw - 1) // tw
    gy = (cam["height"] + th - 1) // th
    toff = sum(((c["width"] + tw - 1) // tw) * ((c["height"] + th - 1) // th) for c in cams[:v])
    ranges = res["ranges"].cpu().numpy().view(np.uint32)[toff:toff + gx * gy].astype(np.int64)
    vals_all = res["vals"].cpu().numpy().view(np.uint32).astype(np.int64)
    # rebase tile lists to a compact per-view array of Gaussian ids
    vals, rr, pos = [], np.zeros_like(ranges), 0
    for t in range(gx * gy):
        s, e = ranges[t]
        seg = vals_all[s:e] - v * n
        vals.append(seg)
        rr[t] = (pos, pos + (e - s)) if e > s else (0, 0)
        pos += e - s
    vals = np.concatenate(vals) if vals else np.zeros(0, np.int64)
    return {
        "rgb": res["rgb"][v].cpu().numpy(),
        "final_T": res["final_T"][v].cpu().numpy(),
        "n_contrib": res["n_contrib"][v].cpu().numpy().view(np.uint32),
        "vals": vals,
        "ranges": rr,
    }


def cuda_sync():
    torch.cuda.synchronize()
