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
    """Integer fields bit-exact outside guard Gaussians; returns a report dict.
    "differ" counts Gaussians with any integer output different (the guard
    items actually taken the other way); each must carry a guard flag."""
    ok = ~guard_mask
    rep = {}
    vis = (o["tiles"] > 0) & (g["tiles"] > 0)
    d_rad = g["radius"] != o["radius"]
    d_til = g["tiles"] != o["tiles"]
    d_rect = np.any(g["rect"] != o["rect"], 1) & vis
    d_dep = g["depth_bits"] != o["depth_bits"]
    rep["radius_mismatch"] = int(np.sum(d_rad & ok))
    rep["tiles_mismatch"] = int(np.sum(d_til & ok))
    rep["rect_mismatch"] = int(np.sum(d_rect & ok))
    rep["depth_mismatch"] = int(np.sum(d_dep & ok))
    rep["differ"] = int(np.sum(d_rad | d_til | d_rect | d_dep))
    rep["in_band"] = int(guard_mask.sum())
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


def _alpha_tile(o_pre, gid, t, W, H, tw, th):
    """FP64 alpha of Gaussian gid over the pixels of tile t (oracle values)."""
    gx = (W + tw - 1) // tw
    ty, tx = divmod(int(t), gx)
    ys, xs = np.mgrid[ty * th:min((ty + 1) * th, H), tx * tw:min((tx + 1) * tw, W)]
    dx = o_pre["uv"][gid, 0] - xs
    dy = o_pre["uv"][gid, 1] - ys
    a, b, c = o_pre["conic"][gid]
    al = np.minimum(0.99, o_pre["opacity"][gid] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
    return ys, xs, al


def image_report(img_g, img_o, exclude):
    """img_*: [3,H,W]. exclude: [H,W] pixels that legitimately took another branch."""
    err = np.abs(img_g.astype(np.float64) - img_o)
    perpix = err.max(0)
    keep = ~exclude
    return {
        "max_abs": float(perpix[keep].max()) if keep.any() else 0.0,
        "max_abs_all": float(perpix.max()),
        "frac_above_fine": float(np.mean(perpix[keep] > IMG_FINE)) if keep.any() else 0.0,
        "n_pix": int(perpix.size),
    }


def assert_image_parity(rep, what=""):
    assert rep["max_abs"] <= IMG_MAX_ABS, (what, rep)
    assert rep["frac_above_fine"] <= IMG_FINE_FRAC, (what, rep)
    assert rep["n_unexplained"] == 0, (what, rep)
    assert rep["n_guard"] <= max(2, GUARD_FRAC * rep["n_pix"]), (what, rep)


def full_view_parity(scene, cam, res_gpu_view, tile, oracle_res=None, tile_mask=None, tight=False):
    """One view of a GPU render (host copies) against the oracle.

    A pixel "disagrees" when its contributor count differs (compared by the
    identity of the last contributor where the two tile lists differ) or its
    colour differs by more than 1e-4. Every disagreeing pixel must be
    explained: an alpha/stop decision on its path lies in the oracle's guard
    band, or a Gaussian present in only one of the two tile lists (a guard
    Gaussian whose rect or radius sits on a decision boundary) reaches
    alpha >= 1/255 there. Disagreeing pixels are the guard items; the image
    tolerance applies to all others."""
    tw, th = tile
    o = oracle_res if oracle_res is not None else oracle.render(scene, cam, tw, th, tile_mask=tile_mask,
                                                                tight=tight)
    W, H = cam["width"], cam["height"]
    g_vals, g_ranges = res_gpu_view["vals"], res_gpu_view["ranges"]
    bad = list_mismatch_tiles(g_vals, g_ranges, o["vals"], o["ranges"])
    if tile_mask is not None:
        bad = np.array([t for t in bad if tile_mask[t]], dtype=np.int64)
    guard_ids = np.nonzero(guard_gaussians(o["pre"]))[0]
    unexplained_tiles = explained_by_guards(bad, o["vals"], o["ranges"], g_vals, g_ranges, guard_ids)
    nc_g = res_gpu_view["n_contrib"].astype(np.int64)
    nc_o = o["n_contrib"].astype(np.int64)
    differ = nc_g != nc_o
    affected = np.zeros((H, W), bool)
    gx = (W + tw - 1) // tw
    for t in bad:
        la = o["vals"][o["ranges"][t][0]:o["ranges"][t][1]]
        lb = g_vals[g_ranges[t][0]:g_ranges[t][1]]
        ty, tx = divmod(int(t), gx)
        sl = (slice(ty * th, min((ty + 1) * th, H)), slice(tx * tw, min((tx + 1) * tw, W)))
        # contributor counts compared by identity of the last contributor
        pa = nc_o[sl]
        pb = nc_g[sl]
        ida = np.where(pa > 0, np.asarray(la, np.int64)[np.maximum(pa - 1, 0)] if len(la) else -1, -1)
        idb = np.where(pb > 0, np.asarray(lb, np.int64)[np.maximum(pb - 1, 0)] if len(lb) else -1, -1)
        differ[sl] = ida != idb
        sym = set(int(x) for x in la) ^ set(int(x) for x in lb)
        if not sym:                                  # same members, order swapped
            affected[sl] = True
        for gid in sym:
            ys, xs, al = _alpha_tile(o["pre"], gid, t, W, H, tw, th)
            affected[ys, xs] |= al >= (1.0 / 255.0) * (1.0 - 1e-3)
    err = np.abs(res_gpu_view["rgb"].astype(np.float64) - o["rgb"]).max(0)
    disagree = differ | (err > 1e-4)
    explained = (o["pguard"] != 0) | affected
    if tile_mask is not None:                    # compare only the sampled tiles' pixels
        sampled = tile_pixel_mask(np.nonzero(tile_mask)[0], W, H, tw, th)
        disagree &= sampled
        rep = image_report(res_gpu_view["rgb"][:, sampled][:, None, :], o["rgb"][:, sampled][:, None, :],
                           disagree[sampled][None, :])
        rep["n_guard"] = int(disagree.sum())
        rep["n_unexplained"] = int((disagree & ~explained).sum())
        rep["n_contrib_mismatch"] = int((differ & ~explained & sampled).sum())
        rep["n_in_band"] = int(((o["pguard"] != 0) & sampled).sum())
        rep["bad_tiles"] = len(bad)
        rep["unexplained_tiles"] = unexplained_tiles
        return rep, o
    rep = image_report(res_gpu_view["rgb"], o["rgb"], disagree)
    rep["n_guard"] = int(disagree.sum())
    rep["n_unexplained"] = int((disagree & ~explained).sum())
    rep["n_contrib_mismatch"] = int((differ & ~explained).sum())
    rep["n_in_band"] = int((o["pguard"] != 0).sum())
    rep["T_max_abs"] = float(np.max(np.abs(res_gpu_view["final_T"] - o["final_T"])[~disagree])) if (~disagree).any() else 0.0
    rep["bad_tiles"] = len(bad)
    rep["unexplained_tiles"] = unexplained_tiles
    return rep, o


def tile_pixel_mask(tiles, W, H, tw, th):
    gx = (W + tw - 1) // tw
    m = np.zeros((H, W), bool)
    for t in tiles:
        ty, tx = divmod(int(t), gx)
        m[ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw] = True
    return m


def sample_tiles(cam, frac, seed, tile=(16, 16)):
    tw, th = tile
    nt = ((cam["width"] + tw - 1) // tw) * ((cam["height"] + th - 1) // th)
    rng = np.random.default_rng(seed)
    mask = np.zeros(nt, np.uint8)
    mask[rng.choice(nt, max(1, int(frac * nt)), replace=False)] = 1
    return mask


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
