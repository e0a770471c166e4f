"""Seeded synthetic scenes and cameras (input data only).

This module draws the Gaussians and cameras that both the CUDA path and the
CPU oracle consume. It holds none of the rasterizer's arithmetic: it only
samples parameter arrays and builds look-at camera matrices, with numpy's
PCG64 generator so that a seed gives the same scene on every host.

The paper evaluates on trained Mip-NeRF 360, Tanks & Templates and Deep
Blending scenes (Sec. IV-A1). None of those are available, so the scenes here
stand in for them with the shapes, sizes and value distributions of the
workloads described in the module-level ``CONFIGS`` table:

* ``tiny``    10,000 Gaussians in a cube, SH degree 0, one 256x256 view.
* ``outdoor`` 500,000 Gaussians, 64 anisotropic clusters plus a 10 % shell at
  radius 10, SH degree 3, 8 orbit views at 1264x832.
* ``indoor``  2.8M Gaussians on the walls of a room box and on interior boxes,
  larger footprints, SH degree 3, one 1332x876 view from inside the room.
* ``batched`` 3M clustered Gaussians, SH degree 3, 64 views of uneven size
  between 800x800 and 1920x1080.
* ``scale``   30M Gaussians in 256 dense clusters plus a sparse background,
  SH degree 3, 16 orbit views at 1920x1080.

Layouts (all float32, C-contiguous):
  means [N,3], scales [N,3] (already exponentiated), quats [N,4] (w,x,y,z,
  unnormalised), opacities [N] (already passed through a sigmoid),
  sh [N,(d+1)^2,3].

A camera is a dict with width, height, fx, fy, cx, cy, viewmat (4x4 row-major
world-to-camera, OpenCV axes: x right, y down, z forward), campos [3] and
bg [3]. Pixel (i, j) is sampled at the integer position (i, j), so the
principal point of a centred camera is ((W-1)/2, (H-1)/2).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1000

CONFIG_INDEX = {"tiny": 0, "outdoor": 1, "indoor": 2, "batched": 3, "scale": 4}


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sh(rng, n, degree, dc_mean=0.5, dc_std=0.2, band_std=0.05):
    k = (degree + 1) ** 2
    sh = np.empty((n, k, 3), dtype=np.float32)
    sh[:, 0, :] = rng.normal(dc_mean, dc_std, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, band_std, size=(n, k - 1, 3))
    return sh


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q *= np.sign(np.diag(r))
    return q


def _clusters(rng, n, n_clusters, centre_lo, centre_hi, spread_lo=0.05, spread_hi=1.0):
    centres = rng.uniform(centre_lo, centre_hi, size=(n_clusters, 3))
    weights = rng.dirichlet(np.full(n_clusters, 0.5))
    counts = rng.multinomial(n, weights)
    pts = np.empty((n, 3), dtype=np.float64)
    pos = 0
    for k in range(n_clusters):
        c = counts[k]
        if c == 0:
            continue
        rot = _random_rotation(rng)
        sd = rng.uniform(spread_lo, spread_hi, size=3)
        local = rng.standard_normal((c, 3)) * sd
        pts[pos:pos + c] = centres[k] + local @ rot.T
        pos += c
    return pts


def look_at(eye, target, width, height, fov_x_deg, bg=(0.0, 0.0, 0.0)):
    """Pinhole camera at ``eye`` looking at ``target`` with world up = +y."""
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    rot = np.stack([right, down, f])
    t = -rot @ eye
    view = np.eye(4)
    view[:3, :3] = rot
    view[:3, 3] = t
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return {
        "width": int(width),
        "height": int(height),
        "fx": float(np.float32(fx)),
        "fy": float(np.float32(fx)),
        "cx": (width - 1) / 2.0,
        "cy": (height - 1) / 2.0,
        "viewmat": view.astype(np.float32),
        "campos": eye.astype(np.float32),
        "bg": np.asarray(bg, dtype=np.float32),
    }


def _orbit(n_views, radius, height, width, img_h, fov=60.0):
    cams = []
    for k in range(n_views):
        th = 2.0 * math.pi * k / n_views
        eye = (radius * math.cos(th), height, radius * math.sin(th))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), width, img_h, fov))
    return cams


def _pack(means, log_scales, quats, opac, sh):
    return {
        "means": np.ascontiguousarray(means, dtype=np.float32),
        "scales": np.ascontiguousarray(np.exp(log_scales), dtype=np.float32),
        "quats": np.ascontiguousarray(quats, dtype=np.float32),
        "opacities": np.ascontiguousarray(opac, dtype=np.float32),
        "sh": np.ascontiguousarray(sh, dtype=np.float32),
    }


def tiny(n=10_000, seed=None, width=256, height=256, sh_degree=0):
    rng = np.random.default_rng(SEED_BASE + 0 if seed is None else seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    log_scales = rng.normal(-4.5, 0.5, size=(n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    sh = _sh(rng, n, sh_degree)
    cams = [look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), width, height, 60.0)]
    return _pack(means, log_scales, quats, opac, sh), cams


def outdoor(n=500_000, seed=None, width=1264, height=832, n_views=8, n_clusters=64):
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    n_shell = n // 10
    n_cl = n - n_shell
    pts = _clusters(rng, n_cl, n_clusters, -4.0, 4.0)
    d = rng.standard_normal((n_shell, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 10.0 * (1.0 + 0.02 * rng.standard_normal(n_shell))
    means = np.concatenate([pts, d * r[:, None]])
    log_scales = rng.normal(-4.0, 0.7, size=(n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    sh = _sh(rng, n, 3)
    cams = _orbit(n_views, 6.0, 1.5, width, height)
    return _pack(means, log_scales, quats, opac, sh), cams


def indoor(n=2_800_000, seed=None, width=1332, height=876, n_patches=1024, n_boxes=32):
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    half = np.array([rng.uniform(3, 6), rng.uniform(1.5, 2.5), rng.uniform(3, 6)])
    n_wall = int(round(0.85 * n))
    n_box = n - n_wall
    # wall patches: pick a wall (axis, side), a patch centre on it, spread in-plane
    axis = rng.integers(0, 3, size=n_patches)
    side = rng.choice([-1.0, 1.0], size=n_patches)
    centres = rng.uniform(-1.0, 1.0, size=(n_patches, 3)) * half
    centres[np.arange(n_patches), axis] = side * half[axis]
    sig = rng.uniform(0.1, 0.6, size=n_patches)
    which = rng.integers(0, n_patches, size=n_wall)
    pts = centres[which] + rng.standard_normal((n_wall, 3)) * sig[which, None]
    a = axis[which]
    pts[np.arange(n_wall), a] = side[which] * half[a] + rng.normal(0.0, 0.02, size=n_wall)
    pts = np.clip(pts, -half, half)
    # interior boxes
    bc = rng.uniform(-0.7, 0.7, size=(n_boxes, 3)) * half
    bh = rng.uniform(0.1, 0.5, size=(n_boxes, 3))
    wb = rng.integers(0, n_boxes, size=n_box)
    bpts = bc[wb] + rng.uniform(-1.0, 1.0, size=(n_box, 3)) * bh[wb]
    means = np.concatenate([pts, bpts])
    log_scales = rng.normal(-3.2, 0.6, size=(n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.5, 1.0, size=n))
    sh = _sh(rng, n, 3)
    az = rng.uniform(0.0, 2.0 * math.pi)
    eye = np.array([0.5 * half[0] * rng.uniform(-1, 1), 0.0, 0.5 * half[2] * rng.uniform(-1, 1)])
    target = eye + np.array([math.cos(az), 0.0, math.sin(az)])
    cams = [look_at(eye, target, width, height, 60.0)]
    return _pack(means, log_scales, quats, opac, sh), cams


def batched(n=3_000_000, seed=None, n_views=64):
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    scene, _ = outdoor(n=n, seed=SEED_BASE + 3 if seed is None else seed, n_views=1)
    cams = []
    for _ in range(n_views):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = math.radians(rng.uniform(-20.0, 40.0))
        r = rng.uniform(5.0, 8.0)
        eye = (r * math.cos(el) * math.cos(az), r * math.sin(el), r * math.cos(el) * math.sin(az))
        w = int(rng.integers(800, 1921))
        h = int(rng.integers(800, 1081))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), w, h, 60.0))
    return scene, cams


def scale(n=30_000_000, seed=None, width=1920, height=1080, n_views=16):
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    n_bg = n // 20
    n_cl = n - n_bg
    pts = _clusters(rng, n_cl, 256, -6.0, 6.0)
    bg = rng.uniform(-20.0, 20.0, size=(n_bg, 3))
    means = np.concatenate([pts, bg])
    log_scales = rng.normal(-4.5, 0.6, size=(n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    sh = _sh(rng, n, 3)
    cams = _orbit(n_views, 8.0, 1.5, width, height)
    return _pack(means, log_scales, quats, opac, sh), cams


CONFIGS = {
    "tiny": tiny,
    "outdoor": outdoor,
    "indoor": indoor,
    "batched": batched,
    "scale": scale,
}


def random_small(n, seed, width=64, height=48, sh_degree=3, opacity_max=None,
                 log_scale_mean=-3.0, log_scale_std=0.5, extent=1.0, dist=3.0):
    """Small random scene for parity and pin tests (a handful of tiles, ragged edges)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, size=(n, 3))
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.0, size=n))
    if opacity_max is not None:
        opac = rng.uniform(0.01, opacity_max, size=n)
    sh = _sh(rng, n, sh_degree, band_std=0.1)
    cam = look_at((0.3, -0.2, -dist), (0.0, 0.0, 0.0), width, height, 60.0)
    return _pack(means, log_scales, quats, opac, sh), [cam]


def crop_camera(cam, x0, y0, w, h):
    """The same camera restricted to the pixel window [x0, x0+w) x [y0, y0+h)."""
    c = dict(cam)
    c["width"] = int(w)
    c["height"] = int(h)
    c["cx"] = cam["cx"] - x0
    c["cy"] = cam["cy"] - y0
    return c
