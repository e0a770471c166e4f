"""FP64 CPU oracle of the Local-GS rasterization path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It is independent of the CUDA library:
it shares no code, header or constant with it, and the product path never
falls back to it.

``render(scene, cam)`` runs the plain definition of 3DGS forward rendering
(Sec. II-A pipeline; Eq. 3DGS alpha; Alg. 1 baseline column) in double
precision and returns every intermediate that the CUDA path also produces,
plus guard flags that mark decisions lying within a guard band of their
threshold (the only places where an FP32 path may legitimately differ in an
integer output).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

# Guard bands (the decision margins inside which an FP32 path may legitimately
# take the other branch): tile-rect edge in px, 3*sqrt(lambda) to an integer
# (relative), near plane (relative), depth float32 rounding midpoint
# (relative; 0 because camera-space z is reproduced bit for bit), det
# (relative), alpha against 1/255 (relative), T(1-alpha) against 1e-4
# (relative), tight-box level tau' (relative) and tight-box span ends (px).
DEFAULT_GUARD = np.array([1e-4, 2e-6, 1e-6, 0.0, 1e-6, 1e-4, 1e-4, 1e-4, 2e-3], dtype=np.float64)

GF_RECT, GF_RADIUS, GF_NEAR, GF_DEPTH, GF_DET, GF_TIGHT = 1, 2, 4, 8, 16, 32

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_sh_basis.restype = ctypes.c_double
        L.orc_sh_basis.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
        L.orc_sh_eval.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_quat_to_rot.argtypes = [_dp, _dp]
        L.orc_cov3d.argtypes = [_dp, _dp, _dp]
        L.orc_ewa.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_preprocess.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                     _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                     _dp, _dp, _u32p, _dp, _i32p, _i32p, _i64p, _dp, _u8p, _u8p]
        L.orc_sort.restype = ctypes.c_int64
        L.orc_sort.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                               ctypes.c_uint32, _i32p, _i64p, _u32p, ctypes.c_int64,
                               _u64p, _u32p, _u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               _dp, _dp, _dp]
        L.orc_tight_rows.restype = ctypes.c_int
        L.orc_tight_rows.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int] * 5 + [ctypes.c_double] * 2 + \
            [_i32p, _i32p, _i32p]
        L.orc_blend.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp,
                                _u32p, _u32p, ctypes.c_int64, _dp, _dp, _dp, _dp, _dp,
                                _dp, _dp, _u32p, _u8p, _u32p, _u32p, _u8p]
        L.orc_blend_literal.argtypes = [ctypes.c_int] * 5 + [_dp, _u32p, _u32p, ctypes.c_int64,
                                                             _dp, _dp, _dp, _dp, _dp, _dp, _dp, _u32p, _u8p]
        L.orc_hoist.argtypes = [ctypes.c_double] * 6 + [_dp]
        L.orc_warp_mask.restype = ctypes.c_uint32
        L.orc_warp_mask.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int] * 5
        L.orc_localgs_pairs.restype = ctypes.c_int64
        L.orc_localgs_pairs.argtypes = [ctypes.c_int] * 5 + [_u32p, _u32p, ctypes.c_int64,
                                                             _dp, _dp, _dp, _u32p]
        L.orc_localgs_pairs_blocks.restype = ctypes.c_int64
        L.orc_localgs_pairs_blocks.argtypes = [ctypes.c_int] * 6 + [_u32p, _u32p, ctypes.c_int64,
                                                                    _dp, _dp, _dp, _u32p]
        L.orc_block_mask.restype = ctypes.c_uint32
        L.orc_block_mask.argtypes = [ctypes.c_double] * 6 + [ctypes.c_int] * 6
        if hasattr(L, "orc_backward"):
            _bind_backward(L)
        _LIB = L
    return _LIB


def _bind_backward(L):
    L.orc_backward.argtypes = [ctypes.c_int64, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                               ctypes.c_int, ctypes.c_int, _dp, _dp,
                               _dp, _dp, _dp, _dp, _dp, _dp]


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a, t):
    return a.ctypes.data_as(t)


def cam_array(cam) -> np.ndarray:
    """Flat 24-double camera: W, H, fx, fy, cx, cy, R[9], t[3], campos[3], bg[3]."""
    v = np.asarray(cam["viewmat"], dtype=np.float64)
    return np.concatenate([
        [cam["width"], cam["height"], float(np.float32(cam["fx"])), float(np.float32(cam["fy"])),
         float(np.float32(cam["cx"])), float(np.float32(cam["cy"]))],
        v[:3, :3].reshape(-1), v[:3, 3], np.asarray(cam["campos"], np.float64),
        np.asarray(cam["bg"], np.float64)]).astype(np.float64)


def _in(x, exact=False):
    """Scene array as float64: the float32 values promoted exactly, or (exact=True,
    for finite differences) the given doubles unchanged."""
    if exact:
        return np.ascontiguousarray(x, dtype=np.float64)
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32), dtype=np.float64)


def sh_degree_of(scene) -> int:
    k = scene["sh"].shape[1]
    return int(round(k ** 0.5)) - 1


def preprocess(scene, cam, tile_w=16, tile_h=16, guard=DEFAULT_GUARD, exact=False, tight=False):
    L = lib()
    n = scene["means"].shape[0]
    deg = sh_degree_of(scene)
    m, s, q, o, sh = (_in(scene[k], exact) for k in ("means", "scales", "quats", "opacities", "sh"))
    c = cam_array(cam)
    g = np.ascontiguousarray(guard, dtype=np.float64)
    out = {
        "uv": np.zeros((n, 2)), "depth": np.zeros(n), "depth_bits": np.zeros(n, np.uint32),
        "conic": np.zeros((n, 3)), "radius": np.zeros(n, np.int32),
        "rect": np.zeros((n, 4), np.int32), "tiles": np.zeros(n, np.int64),
        "rgb": np.zeros((n, 3)), "clamped": np.zeros((n, 3), np.uint8),
        "gflags": np.zeros(n, np.uint8),
    }
    L.orc_preprocess(n, deg, _p(m, _dp), _p(s, _dp), _p(q, _dp), _p(o, _dp), _p(sh, _dp),
                     _p(c, _dp), tile_w, tile_h, int(bool(tight)), _p(g, _dp),
                     _p(out["uv"], _dp), _p(out["depth"], _dp), _p(out["depth_bits"], _u32p),
                     _p(out["conic"], _dp), _p(out["radius"], _i32p), _p(out["rect"], _i32p),
                     _p(out["tiles"], _i64p), _p(out["rgb"], _dp), _p(out["clamped"], _u8p),
                     _p(out["gflags"], _u8p))
    out["opacity"] = o
    out["tight"] = bool(tight)
    return out


def sort(pre, cam, tile_w=16, tile_h=16, tile_offset=0, val_offset=0):
    """Duplicate + stable sort; tight-box emission when pre came from
    preprocess(..., tight=True)."""
    L = lib()
    W, H = cam["width"], cam["height"]
    gx, gy = (W + tile_w - 1) // tile_w, (H + tile_h - 1) // tile_h
    n = pre["tiles"].shape[0]
    K = int(pre["tiles"].sum())
    keys = np.zeros(max(K, 1), np.uint64)
    vals = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros((gx * gy, 2), np.uint32)
    tight = bool(pre.get("tight", False))
    r = L.orc_sort(n, gx, gy, tile_offset, val_offset, _p(pre["rect"], _i32p),
                   _p(pre["tiles"], _i64p), _p(pre["depth_bits"], _u32p), K,
                   _p(keys, _u64p), _p(vals, _u32p), _p(ranges, _u32p), int(tight), tile_w, tile_h,
                   _p(np.ascontiguousarray(pre["uv"]), _dp), _p(np.ascontiguousarray(pre["conic"]), _dp),
                   _p(np.ascontiguousarray(pre["opacity"]), _dp))
    assert 0 <= r <= K and (tight or r == K)
    return keys[:r], vals[:r], ranges


def blend(pre, vals, ranges, cam, tile_w=16, tile_h=16, guard=DEFAULT_GUARD, tile_mask=None):
    L = lib()
    W, H = cam["width"], cam["height"]
    bg = np.asarray(cam["bg"], np.float64)
    out_rgb = np.zeros((3, H, W))
    final_T = np.zeros((H, W))
    n_contrib = np.zeros((H, W), np.uint32)
    pguard = np.zeros((H, W), np.uint8)
    stop_pos = np.zeros((H, W), np.uint32)
    n_useful = np.zeros((H, W), np.uint32)
    v = np.ascontiguousarray(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    g = np.ascontiguousarray(guard, dtype=np.float64)
    L.orc_blend(W, H, tile_w, tile_h, _p(bg, _dp), _p(v, _u32p), _p(ranges, _u32p), 0,
                _p(pre["uv"], _dp), _p(pre["conic"], _dp), _p(pre["opacity"], _dp),
                _p(pre["rgb"], _dp), _p(g, _dp), _p(out_rgb, _dp), _p(final_T, _dp),
                _p(n_contrib, _u32p), _p(pguard, _u8p), _p(stop_pos, _u32p), _p(n_useful, _u32p),
                None if tile_mask is None else _p(np.ascontiguousarray(tile_mask, np.uint8), _u8p))
    return {"rgb": out_rgb, "final_T": final_T, "n_contrib": n_contrib, "pguard": pguard,
            "stop_pos": stop_pos, "n_useful": n_useful}


def blend_literal(pre, vals, ranges, cam, tile_w=16, tile_h=16, guard=DEFAULT_GUARD, n_warps=8):
    """Paper-literal warp-coherent blending (no per-pixel stop or 1/255 test)."""
    L = lib()
    W, H = cam["width"], cam["height"]
    bg = np.asarray(cam["bg"], np.float64)
    out_rgb = np.zeros((3, H, W))
    final_T = np.zeros((H, W))
    n_contrib = np.zeros((H, W), np.uint32)
    pguard = np.zeros((H, W), np.uint8)
    v = np.ascontiguousarray(vals, np.uint32) if len(vals) else np.zeros(1, np.uint32)
    g = np.ascontiguousarray(guard, dtype=np.float64)
    L.orc_blend_literal(W, H, tile_w, tile_h, n_warps, _p(bg, _dp), _p(v, _u32p), _p(ranges, _u32p), 0,
                        _p(pre["uv"], _dp), _p(pre["conic"], _dp), _p(pre["opacity"], _dp),
                        _p(pre["rgb"], _dp), _p(g, _dp), _p(out_rgb, _dp), _p(final_T, _dp),
                        _p(n_contrib, _u32p), _p(pguard, _u8p))
    return {"rgb": out_rgb, "final_T": final_T, "n_contrib": n_contrib, "pguard": pguard}


def render(scene, cam, tile_w=16, tile_h=16, guard=DEFAULT_GUARD, exact=False, tile_mask=None,
           tight=False, literal=False):
    """Full forward pass for one view: preprocess, sort, blend (optionally only
    the pixels of the tiles selected by tile_mask; tight-box emission with
    tight=True; the paper-literal blending with literal=True)."""
    pre = preprocess(scene, cam, tile_w, tile_h, guard, exact, tight)
    keys, vals, ranges = sort(pre, cam, tile_w, tile_h)
    if literal:
        img = blend_literal(pre, vals, ranges, cam, tile_w, tile_h, guard)
    else:
        img = blend(pre, vals, ranges, cam, tile_w, tile_h, guard, tile_mask)
    img.update({"pre": pre, "keys": keys, "vals": vals, "ranges": ranges})
    return img


def hoist(a, b, c, o, dx, dy):
    V = np.zeros(6)
    lib().orc_hoist(a, b, c, o, dx, dy, _p(V, _dp))
    return V


def warp_mask(a, b, c, o, mux, muy, X0, Y0, tile_w=16, tile_h=16, n_warps=8):
    return int(lib().orc_warp_mask(a, b, c, o, mux, muy, X0, Y0, tile_w, tile_h, n_warps))


def tight_rows(a, b, c, o, mux, muy, X0, ry0, ry1, tile_w=16, tile_h=16, band_tau=0.0, band_px=0.0):
    """Kept tile rows (lo, hi, count, guard) of one column strip under the
    tight-box emission rule."""
    lo, hi, gd = ctypes.c_int32(0), ctypes.c_int32(-1), ctypes.c_int32(0)
    k = lib().orc_tight_rows(a, b, c, o, mux, muy, X0, tile_w, tile_h, ry0, ry1, band_tau, band_px,
                             ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(gd))
    return lo.value, hi.value, int(k), bool(gd.value)


def block_mask(a, b, c, o, mux, muy, X0, Y0, tile_w=16, tile_h=16, block_w=16, block_h=2):
    """Mask of (tile_w/block_w) x (tile_h/block_h) warp blocks, bit by*nbx + bx."""
    return int(lib().orc_block_mask(a, b, c, o, mux, muy, X0, Y0, tile_w, tile_h, block_w, block_h))


def localgs_pairs(res, cam, tile_w=16, tile_h=16, n_warps=8, block=None):
    """Pixel-Gaussian pairs of the Local-GS schedule (warp mask + warp exit);
    block = (block_w, block_h) of one warp, None = n_warps full-width strips."""
    pre = res["pre"]
    W, H = cam["width"], cam["height"]
    bw, bh = (tile_w, tile_h // n_warps) if block is None else block
    v = np.ascontiguousarray(res["vals"], np.uint32) if len(res["vals"]) else np.zeros(1, np.uint32)
    return int(lib().orc_localgs_pairs_blocks(W, H, tile_w, tile_h, bw, bh, _p(v, _u32p),
                                              _p(res["ranges"], _u32p), 0, _p(pre["uv"], _dp),
                                              _p(pre["conic"], _dp), _p(pre["opacity"], _dp),
                                              _p(np.ascontiguousarray(res["stop_pos"]), _u32p)))


def backward(scene, cam, dL_drgb, dL_dT=None, tile_w=16, tile_h=16, exact=False):
    """Hand adjoint of render() for L = <dL_drgb, rgb> + <dL_dT, final_T>.
    Returns gradients w.r.t. means, scales, quats, opacities, sh and the 2D
    per-Gaussian gradients g2d [N, 9] = dL/d(u, v, a, b, c, o, r, g, b)."""
    L = lib()
    n = scene["means"].shape[0]
    deg = sh_degree_of(scene)
    m, s, q, o, sh = (_in(scene[k], exact) for k in ("means", "scales", "quats", "opacities", "sh"))
    c = cam_array(cam)
    g = np.ascontiguousarray(dL_drgb, np.float64)
    gT = None if dL_dT is None else np.ascontiguousarray(dL_dT, np.float64)
    out = {"means": np.zeros((n, 3)), "scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
           "opacities": np.zeros(n), "sh": np.zeros(sh.shape), "g2d": np.zeros((n, 9))}
    L.orc_backward(n, deg, _p(m, _dp), _p(s, _dp), _p(q, _dp), _p(o, _dp), _p(sh, _dp), _p(c, _dp),
                   tile_w, tile_h, _p(g, _dp), None if gT is None else _p(gT, _dp),
                   _p(out["means"], _dp), _p(out["scales"], _dp), _p(out["quats"], _dp),
                   _p(out["opacities"], _dp), _p(out["sh"], _dp), _p(out["g2d"], _dp))
    return out


def sh_basis(l, m, d):
    d = np.ascontiguousarray(d, np.float64)
    return float(lib().orc_sh_basis(l, m, _p(d, _dp)))


def quat_to_rot(q):
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9)
    lib().orc_quat_to_rot(_p(q, _dp), _p(R, _dp))
    return R.reshape(3, 3)


def cov3d(s, q):
    s = np.ascontiguousarray(s, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    S = np.zeros(9)
    lib().orc_cov3d(_p(s, _dp), _p(q, _dp), _p(S, _dp))
    return S.reshape(3, 3)


def ewa(cam, t, Sig):
    c = cam_array(cam)
    t = np.ascontiguousarray(t, np.float64)
    Sig = np.ascontiguousarray(Sig, np.float64).reshape(-1)
    out = np.zeros(3)
    lib().orc_ewa(_p(c, _dp), _p(t, _dp), _p(Sig, _dp), _p(out, _dp))
    return out


__all__ = ["render", "backward", "preprocess", "sort", "blend", "blend_literal", "hoist", "warp_mask",
           "block_mask", "tight_rows",
           "localgs_pairs",
           "sh_basis", "quat_to_rot", "cov3d", "ewa", "num_threads", "cam_array",
           "DEFAULT_GUARD"]
os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")
