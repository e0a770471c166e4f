"""Python binding of the Local-GS rasterizer with the C ABI's names.

Each function marshals torch CUDA tensors into the structures of include/lgs.h
and calls the CUDA library on the current torch stream; no arithmetic of the
rasterizer happens here. Buffers are allocated by torch (the library never
allocates), so repeated calls can reuse them (see ``Frame``).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

_TILES = {(16, 16), (8, 32), (32, 8), (32, 32), (16, 32), (32, 16)}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# warp blocks of the Local-GS render per tile shape (the first is the default:
# the paper's layout for 256-pixel tiles; larger tiles are rendered as 16x16
# regions of 8x8 blocks)
WARP_BLOCKS = {(16, 16): ((16, 2), (8, 4), (16, 4), (8, 8)), (8, 32): ((8, 4), (8, 8)),
               (32, 8): ((32, 1), (8, 8)), (32, 32): ((8, 8),), (16, 32): ((8, 8),), (32, 16): ((8, 8),)}


def config(tile=(16, 16), mode="localgs", flags=0, batch=0, block=None) -> L.lgs_config:
    """lgs_config; block = (warp_w, warp_h) of the Local-GS render, None = the
    paper's full-width strips."""
    if tuple(tile) not in _TILES:
        raise ValueError(f"tile shape {tile} not in {_TILES}")
    m = {"localgs": L.MODE_LOCALGS, "plain": L.MODE_PLAIN, "literal": L.MODE_LITERAL,
         "global": L.MODE_GLOBAL}[mode]
    wx, wy = (0, 0) if block is None else (int(block[0]), int(block[1]))
    return L.lgs_config(int(tile[0]), int(tile[1]), m, int(batch), int(flags), wx, wy)


def with_flags(cfg: L.lgs_config, flags) -> L.lgs_config:
    """A copy of cfg with other flags."""
    return L.lgs_config(cfg.tile_w, cfg.tile_h, cfg.mode, cfg.batch, int(flags), cfg.warp_w, cfg.warp_h)


def cameras(cams) -> ctypes.Array:
    """ctypes array of lgs_camera from camera dicts (see scenes.look_at)."""
    if not 1 <= len(cams) <= L.LGS_MAX_VIEWS:
        raise ValueError(f"1..{L.LGS_MAX_VIEWS} views per call")
    arr = (L.lgs_camera * len(cams))()
    for i, c in enumerate(cams):
        a = arr[i]
        a.width, a.height = int(c["width"]), int(c["height"])
        a.fx, a.fy, a.cx, a.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
        vm = np.asarray(c["viewmat"], np.float32).reshape(-1)
        for k in range(16):
            a.viewmat[k] = float(vm[k])
        for k in range(3):
            a.campos[k] = float(c["campos"][k])
            a.bg[k] = float(c["bg"][k])
    return arr


def to_device(scene: dict, device="cuda") -> dict:
    """Scene arrays (numpy or torch) as contiguous float32 device tensors."""
    out = {}
    for k in ("means", "scales", "quats", "opacities", "sh"):
        v = scene[k]
        t = v if isinstance(v, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(v))
        out[k] = t.to(device=device, dtype=torch.float32).contiguous()
    return out


def gaussians(g: dict) -> L.lgs_gaussians:
    n = g["means"].shape[0]
    k = g["sh"].shape[1] if n else 1
    deg = int(round(k ** 0.5)) - 1
    return L.lgs_gaussians(n, deg, g["means"].data_ptr(), g["scales"].data_ptr(),
                           g["quats"].data_ptr(), g["opacities"].data_ptr(), g["sh"].data_ptr())


def new_status(device="cuda") -> torch.Tensor:
    return torch.zeros(L.LGS_STATUS_WORDS, dtype=torch.int64, device=device)


@dataclass
class PreOut:
    """Per-(view, Gaussian) outputs of lgs_preprocess (M = views * N rows)."""
    xy: torch.Tensor       # [M,4] f32 (u_hi, v_hi, u_lo, v_lo)
    conic: torch.Tensor    # [M,4] f32 (a, b, c, o)
    rgb: torch.Tensor      # [M,4] f32 (r, g, b, depth)
    depth: torch.Tensor    # [M] f32
    radius: torch.Tensor   # [M] i32
    tiles: torch.Tensor    # [M] i32 storage of u32
    rect: torch.Tensor     # [M] i64 storage of u64
    flags: torch.Tensor    # [M] u8
    emit: torch.Tensor = None  # [M,8] i32 storage of u32: emission records (optional)

    @staticmethod
    def empty(m, device="cuda", emit=True):
        f = dict(device=device)
        return PreOut(torch.empty((m, 4), dtype=torch.float32, **f),
                      torch.empty((m, 4), dtype=torch.float32, **f),
                      torch.empty((m, 4), dtype=torch.float32, **f),
                      torch.empty(m, dtype=torch.float32, **f),
                      torch.empty(m, dtype=torch.int32, **f),
                      torch.empty(m, dtype=torch.int32, **f),
                      torch.empty(m, dtype=torch.int64, **f),
                      torch.empty(m, dtype=torch.uint8, **f),
                      torch.empty((m, 8), dtype=torch.int32, **f) if emit else None)

    def rows(self, a, b) -> "PreOut":
        """The entries a..b-1 (e.g. the views of a group), as views of the same memory."""
        return PreOut(*(t[a:b] if t is not None else None
                        for t in (self.xy, self.conic, self.rgb, self.depth, self.radius, self.tiles,
                                  self.rect, self.flags, self.emit)))

    def struct(self) -> L.lgs_pre_out:
        return L.lgs_pre_out(*(t.data_ptr() if t is not None else None
                               for t in (self.xy, self.conic, self.rgb, self.depth, self.radius,
                                         self.tiles, self.rect, self.flags, self.emit)))


def preprocess(g, cams, cfg, out=None, status=None, stream=None) -> PreOut:
    carr = cams if isinstance(cams, ctypes.Array) else cameras(cams)
    n = g["means"].shape[0]
    m = n * len(carr)
    out = out if out is not None else PreOut.empty(max(m, 1), g["means"].device)
    status = status if status is not None else new_status(g["means"].device)
    gs = gaussians(g)
    ps = out.struct()
    L.check(L.load().lgs_preprocess(ctypes.byref(gs), carr, len(carr), ctypes.byref(cfg),
                                    ctypes.byref(ps), _ptr(status), _stream(stream)),
            "lgs_preprocess")
    return out


def sort_workspace_size(m, capacity) -> int:
    return int(L.load().lgs_sort_workspace_size(int(m), int(capacity)))


def n_tiles(cams, cfg) -> int:
    return sum(((c["width"] + cfg.tile_w - 1) // cfg.tile_w) * ((c["height"] + cfg.tile_h - 1) // cfg.tile_h)
               for c in cams)


def n_pixels(cams) -> int:
    return sum(int(c["width"]) * int(c["height"]) for c in cams)


def sort(pre: PreOut, n, cams, cfg, capacity, keys=None, vals=None, ranges=None, workspace=None,
         status=None, stream=None, with_keys=True):
    """lgs_sort. with_keys=False passes NULL keys: only values and ranges are written."""
    carr = cameras(cams)
    dev = pre.xy.device
    m = n * len(cams)
    if with_keys and keys is None:
        keys = torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    vals = vals if vals is not None else torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    ranges = ranges if ranges is not None else torch.empty((n_tiles(cams, cfg), 2), dtype=torch.int32,
                                                           device=dev)
    ws_bytes = sort_workspace_size(m, capacity)
    workspace = workspace if workspace is not None else torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    status = status if status is not None else new_status(dev)
    ps = pre.struct()
    L.check(L.load().lgs_sort(ctypes.byref(ps), n, carr, len(carr), ctypes.byref(cfg), capacity,
                              _ptr(keys), _ptr(vals), _ptr(ranges), _ptr(workspace), ws_bytes,
                              _ptr(status), _stream(stream)), "lgs_sort")
    return keys, vals, ranges


def sort_static(pre: PreOut, n, cams, cfg, capacity, keys=None, vals=None, ranges=None,
                status=None, stream=None):
    """lgs_sort_static: the sort with the library's static scratch (no workspace)."""
    carr = cameras(cams)
    dev = pre.xy.device
    keys = keys if keys is not None else torch.empty(max(capacity, 1), dtype=torch.int64, device=dev)
    vals = vals if vals is not None else torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    ranges = ranges if ranges is not None else torch.empty((n_tiles(cams, cfg), 2), dtype=torch.int32,
                                                           device=dev)
    status = status if status is not None else new_status(dev)
    ps = pre.struct()
    L.check(L.load().lgs_sort_static(ctypes.byref(ps), n, carr, len(carr), ctypes.byref(cfg), capacity,
                                     _ptr(keys), _ptr(vals), _ptr(ranges), _ptr(status),
                                     _stream(stream)), "lgs_sort_static")
    return keys, vals, ranges


def render_fwd(pre: PreOut, vals, ranges, cams, cfg, rgb=None, final_T=None, n_contrib=None,
               status=None, stream=None):
    carr = cameras(cams)
    dev = pre.xy.device
    P = n_pixels(cams)
    rgb = rgb if rgb is not None else torch.empty(3 * P, dtype=torch.float32, device=dev)
    final_T = final_T if final_T is not None else torch.empty(P, dtype=torch.float32, device=dev)
    n_contrib = n_contrib if n_contrib is not None else torch.empty(P, dtype=torch.int32, device=dev)
    status = status if status is not None else new_status(dev)
    ps = pre.struct()
    L.check(L.load().lgs_render_fwd(ctypes.byref(ps), _ptr(vals), _ptr(ranges), carr, len(carr),
                                    ctypes.byref(cfg), _ptr(rgb), _ptr(final_T), _ptr(n_contrib),
                                    _ptr(status), _stream(stream)), "lgs_render_fwd")
    return rgb, final_T, n_contrib


def new_grads(g, n_views):
    """Zeroed gradient buffers for lgs_render_bwd (3D grads + 2D scratch)."""
    dev = g["means"].device
    n = g["means"].shape[0]
    m = max(n * n_views, 1)
    z = lambda *s: torch.zeros(*s, dtype=torch.float32, device=dev)
    return {"means": z(g["means"].shape), "scales": z(g["scales"].shape), "quats": z(g["quats"].shape),
            "opacities": z(g["opacities"].shape), "sh": z(g["sh"].shape),
            "xy2d": z((m, 2)), "conic2d": z((m, 4)), "rgb2d": z((m, 4))}


def render_bwd(g, cams, cfg, pre: PreOut, vals, ranges, final_T, n_contrib, dL_drgb, dL_dT=None,
               grads=None, status=None, stream=None):
    """lgs_render_bwd: gradients of <dL_drgb, rgb> + <dL_dT, final_T>."""
    carr = cameras(cams)
    grads = grads if grads is not None else new_grads(g, len(cams))
    status = status if status is not None else new_status(g["means"].device)
    gs = gaussians(g)
    ps = pre.struct()
    gr = L.lgs_grads(*(grads[k].data_ptr() for k in ("means", "scales", "quats", "opacities", "sh",
                                                      "xy2d", "conic2d", "rgb2d")))
    L.check(L.load().lgs_render_bwd(ctypes.byref(gs), carr, len(carr), ctypes.byref(cfg), ctypes.byref(ps),
                                    _ptr(vals), _ptr(ranges), _ptr(final_T), _ptr(n_contrib),
                                    _ptr(dL_drgb.contiguous()),
                                    _ptr(None if dL_dT is None else dL_dT.contiguous()),
                                    ctypes.byref(gr), _ptr(status), _stream(stream)), "lgs_render_bwd")
    return grads


class RenderFunction(torch.autograd.Function):
    """Differentiable forward render of a batch of views.

    forward(means, scales, quats, opacities, sh, cams, tile, flags) -> (rgb, final_T),
    both flat over the views (see include/lgs.h); backward runs lgs_render_bwd
    from the saved preprocess outputs, tile lists, final_T and n_contrib.
    """

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, cams, tile=(16, 16), flags=0):
        g = {"means": means.contiguous(), "scales": scales.contiguous(), "quats": quats.contiguous(),
             "opacities": opacities.contiguous(), "sh": sh.contiguous()}
        res = render(g, cams, tile=tile, flags=flags)
        ctx.cams, ctx.cfg, ctx.g = cams, res["cfg"], g
        ctx.pre = res["pre"]
        ctx.save_for_backward(res["vals"], res["ranges"], res["T_flat"], res["nc_flat"])
        return res["rgb_flat"], res["T_flat"]

    @staticmethod
    def backward(ctx, d_rgb, d_T):
        vals, ranges, T, nc = ctx.saved_tensors
        gr = render_bwd(ctx.g, ctx.cams, ctx.cfg, ctx.pre, vals, ranges, T, nc, d_rgb.contiguous(),
                        None if d_T is None else d_T.contiguous())
        return gr["means"], gr["scales"], gr["quats"], gr["opacities"], gr["sh"], None, None, None


def selftest_wait_timeout(spin_limit=1000, status=None, stream=None) -> np.ndarray:
    """Makes one bounded device wait run out (lgs_selftest_wait_timeout) and
    returns the status words it leaves."""
    dev = torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty(L.SELFTEST_WORKSPACE_BYTES, dtype=torch.uint8, device=dev)
    status = status if status is not None else new_status(dev)
    L.check(L.load().lgs_selftest_wait_timeout(int(spin_limit), _ptr(ws), ws.numel(), _ptr(status),
                                               _stream(stream)), "lgs_selftest_wait_timeout")
    return read_status(status, stream)


def get_device_status(status, stream=None):
    """(code, detail) of the first device-side error recorded in `status`
    (lgs_get_device_status; synchronises the stream)."""
    code, detail = ctypes.c_int32(0), ctypes.c_int64(0)
    L.check(L.load().lgs_get_device_status(_ptr(status), _stream(stream), ctypes.byref(code),
                                           ctypes.byref(detail)), "lgs_get_device_status")
    return int(code.value), int(detail.value)


def read_status(status, stream=None) -> np.ndarray:
    h = (ctypes.c_int64 * L.LGS_STATUS_WORDS)()
    L.check(L.load().lgs_read_status(_ptr(status), h, _stream(stream)), "lgs_read_status")
    return np.array(h[:], dtype=np.int64)


def split_views(flat, cams, channels):
    """Views of a concatenated per-pixel output as a list of [C,H,W] / [H,W] tensors."""
    out, off = [], 0
    for c in cams:
        hw = int(c["width"]) * int(c["height"])
        if channels:
            out.append(flat[channels * off: channels * (off + hw)].view(channels, c["height"], c["width"]))
        else:
            out.append(flat[off: off + hw].view(c["height"], c["width"]))
        off += hw
    return out


def render(g, cams, tile=(16, 16), mode="localgs", capacity=None, flags=0, stream=None):
    """Forward pass for a batch of views: preprocess, sort, render.

    If ``capacity`` is None the instance buffers are sized from the count the
    sort reports (one status read), retrying once when a first guess is short.
    Returns a dict with the per-view images and every intermediate.
    """
    cfg = config(tile, mode, flags)
    n = g["means"].shape[0]
    status = new_status(g["means"].device)
    pre = preprocess(g, cams, cfg, status=status, stream=stream)
    cap = capacity if capacity is not None else max(1 << 16, 4 * n * len(cams))
    keys, vals, ranges = sort(pre, n, cams, cfg, cap, status=status, stream=stream)
    st = read_status(status, stream)
    if st[L.ST_CODE] == L.LGS_ERR_CAPACITY:
        if capacity is not None:
            raise L.LgsError(L.LGS_ERR_CAPACITY, f"lgs_sort needs capacity {st[L.ST_DETAIL]}")
        cap = int(st[L.ST_DETAIL])
        status.zero_()
        keys, vals, ranges = sort(pre, n, cams, cfg, cap, status=status, stream=stream)
        st = read_status(status, stream)
    if st[L.ST_CODE] != 0:
        raise L.LgsError(int(st[L.ST_CODE]), "device status")
    K = int(st[L.ST_NUM_INSTANCES])
    rgb, T, nc = render_fwd(pre, vals, ranges, cams, cfg, status=status, stream=stream)
    return {"rgb": split_views(rgb, cams, 3), "final_T": split_views(T, cams, 0),
            "n_contrib": split_views(nc, cams, 0), "rgb_flat": rgb, "T_flat": T, "nc_flat": nc,
            "pre": pre, "keys": keys[:K], "vals": vals[:K], "ranges": ranges, "K": K,
            "status": status, "cfg": cfg}
