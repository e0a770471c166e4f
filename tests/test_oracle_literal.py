"""Pins of the oracle's paper-literal blending (Alg. 1 right column read
literally: warp-mask culling only, w = alpha T, T -= w, warp-level exit)."""
import math

import numpy as np

import oracle
from paper_2606_16566_gb300 import scenes

from test_oracle_tight import _sampled_span


def _strip_hit(a, b, c, o, mux, muy, X0, tw, r0, r1):
    """Brute-force mask bit: do the pixel rows r0..r1-1 meet the widened span
    (dense sampling of the column strip, no case analysis)?"""
    tau = 1.001 * 2 * math.log(255 * o) + 0.02
    if tau <= 0:
        return False
    sp = _sampled_span(a, b, c, tau, X0 - mux, X0 + tw - 1 - mux)
    if sp is None:
        return False
    P = math.ceil(muy + sp[0] - 1 / 64)
    Q = math.floor(muy + sp[1] + 1 / 64)
    return max(r0, P) <= min(r1 - 1, Q)


def _brute_literal(pre, vals, ranges, W, H, tw=16, th=16, nw=8, bg=(0, 0, 0)):
    rows = th // nw
    gx, gy = (W + tw - 1) // tw, (H + th - 1) // th
    img = np.zeros((3, H, W))
    TT = np.ones((H, W))
    nc = np.zeros((H, W), np.int64)
    for ty in range(gy):
        for tx in range(gx):
            s, e = ranges[ty * gx + tx]
            for w in range(nw):
                X0, Y0 = tx * tw, ty * th + w * rows
                pix = [(x, y) for y in range(Y0, Y0 + rows) for x in range(X0, X0 + tw) if x < W and y < H]
                if not pix:
                    continue
                T = {p: 1.0 for p in pix}
                C = {p: np.zeros(3) for p in pix}
                last = 0
                for k in range(s, e):
                    i = int(vals[k])
                    a, b, c = pre["conic"][i]
                    o = float(pre["opacity"][i])
                    mux, muy = pre["uv"][i]
                    if not _strip_hit(a, b, c, o, mux, muy, X0, tw, Y0, Y0 + rows):
                        continue
                    if max(T.values()) < 1e-4:
                        break
                    for p in pix:
                        dx, dy = mux - p[0], muy - p[1]
                        al = min(0.99, o * math.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
                        wgt = al * T[p]
                        C[p] += pre["rgb"][i] * wgt
                        T[p] -= wgt
                    last = k - s + 1
                for p in pix:
                    img[:, p[1], p[0]] = C[p] + T[p] * np.asarray(bg)
                    TT[p[1], p[0]] = T[p]
                    nc[p[1], p[0]] = last
    return img, TT, nc


def test_literal_equals_bruteforce_per_strip():
    sc, cams = scenes.random_small(80, seed=61, width=48, height=40)
    cam = dict(cams[0])
    cam["bg"] = np.array([0.2, 0.5, 0.1], np.float32)
    r = oracle.render(sc, cam, literal=True)
    img, TT, nc = _brute_literal(r["pre"], r["vals"], r["ranges"], 48, 40,
                                 bg=np.asarray(cam["bg"], np.float64))
    skip = r["pguard"] != 0           # sampled-span ties within the guard band
    assert skip.mean() < 0.1
    np.testing.assert_allclose(r["rgb"][:, ~skip], img[:, ~skip], atol=1e-12)
    np.testing.assert_allclose(r["final_T"][~skip], TT[~skip], atol=1e-12)
    assert np.array_equal(r["n_contrib"][~skip].astype(np.int64), nc[~skip])


def test_literal_conserves_energy_for_white_gaussians():
    """With every colour 1 and a black background, C = 1 - T in every channel:
    each step moves exactly w from T to C."""
    sc, cams = scenes.random_small(300, seed=62, width=90, height=70)
    sc["sh"][:] = 0.0
    sc["sh"][:, 0, :] = 0.5 / 0.28209479177387814          # rgb = Y00 * sh + 0.5 = 1
    cam = dict(cams[0])
    cam["bg"] = np.zeros(3, np.float32)
    r = oracle.render(sc, cam, literal=True)
    assert np.allclose(r["pre"]["rgb"][r["pre"]["tiles"] > 0], 1.0, atol=1e-6)
    for ch in range(3):
        np.testing.assert_allclose(r["rgb"][ch], 1.0 - r["final_T"], atol=1e-5)


def test_literal_warp_exit_after_opaque_stack():
    """Coincident wide Gaussians of alpha ~0.95 over a strip: T ~ 5e-2, 2.5e-3,
    1.26e-4, 6.3e-6. The strip is not done after three (1.26e-4 >= 1e-4),
    processes the fourth, and leaves before the fifth: n_contrib = 4."""
    n = 6
    cam = scenes.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32, 60.0)
    sc = {"means": np.zeros((n, 3), np.float32), "scales": np.full((n, 3), 20.0, np.float32),
          "quats": np.tile(np.float32([1, 0, 0, 0]), (n, 1)), "opacities": np.full(n, 0.95, np.float32),
          "sh": np.full((n, 1, 3), 0.3, np.float32)}
    sc["means"][:, 2] = np.arange(n, dtype=np.float32) * 1e-3      # distinct depths, front to back
    r = oracle.render(sc, cam, literal=True)
    strip = (slice(14, 16), slice(16, 32))
    assert np.all(r["n_contrib"][strip] == 4)
    assert np.all(r["final_T"][strip] < 1e-4) and np.all(r["final_T"][strip] > 1e-6)
    assert not r["pguard"][strip].any()


def test_literal_single_gaussian_closed_form():
    """One Gaussian: a pixel of a strip whose mask bit is set gets f alpha +
    (1 - alpha) bg even where alpha < 1/255; other pixels keep the background."""
    sc, cams = scenes.random_small(1, seed=63, width=64, height=64)
    sc["means"][:] = 0.0
    cam = dict(cams[0])
    cam["bg"] = np.array([0.1, 0.2, 0.3], np.float32)
    r = oracle.render(sc, cam, literal=True)
    pre = r["pre"]
    a, b, c = pre["conic"][0]
    o = float(pre["opacity"][0])
    mux, muy = pre["uv"][0]
    ys, xs = np.mgrid[0:64, 0:64]
    dx, dy = mux - xs, muy - ys
    al = np.minimum(0.99, o * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
    bg = np.asarray(cam["bg"], np.float64)
    x0, y0, x1, y1 = pre["rect"][0]
    n_small = 0
    for ty in range(4):
        for tx in range(4):
            for w in range(8):
                Y0 = ty * 16 + 2 * w
                sl = (slice(Y0, Y0 + 2), slice(tx * 16, tx * 16 + 16))
                inside = (x0 <= tx < x1 and y0 <= ty < y1 and
                          _strip_hit(a, b, c, o, mux, muy, tx * 16, 16, Y0, Y0 + 2))
                for ch in range(3):
                    ref = (pre["rgb"][0, ch] * al[sl] + (1 - al[sl]) * bg[ch]) if inside else bg[ch]
                    np.testing.assert_allclose(r["rgb"][ch][sl], ref, atol=1e-12)
                if inside:
                    n_small += int(np.sum(al[sl] < 1 / 255))
    assert n_small > 0                  # the literal form blends sub-threshold alphas
