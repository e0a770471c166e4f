"""Pins of the FP64 oracle against facts other than itself.

Each test checks the oracle against a closed form, a textbook value, a brute
force computation written independently here, or finite differences, so that
a dropped term, a wrong sign or index, or a transposed operand in the oracle
fails one of them. CPU only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_16566_gb300 import scenes


def _axis_camera(W, H, f, bg=(0.0, 0.0, 0.0)):
    return {"width": W, "height": H, "fx": f, "fy": f, "cx": (W - 1) / 2.0, "cy": (H - 1) / 2.0,
            "viewmat": np.eye(4, dtype=np.float32), "campos": np.zeros(3, np.float32),
            "bg": np.asarray(bg, np.float32)}


def _scene(means, scales, quats, opac, sh):
    return {"means": np.asarray(means, np.float32), "scales": np.asarray(scales, np.float32),
            "quats": np.asarray(quats, np.float32), "opacities": np.asarray(opac, np.float32),
            "sh": np.asarray(sh, np.float32)}


Y00 = 0.5 / math.sqrt(math.pi)


# --------------------------------------------------------------------------- geometry
def test_quaternion_convention():
    # a rotation by +90 degrees about z maps e_x to e_y
    c = math.cos(math.pi / 4)
    R = oracle.quat_to_rot([c, 0.0, 0.0, c])
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-15)
    # unnormalised input is normalised first
    np.testing.assert_allclose(oracle.quat_to_rot([2 * c, 0, 0, 2 * c]), R, atol=1e-15)
    # a rotation by +90 degrees about x maps e_y to e_z
    Rx = oracle.quat_to_rot([c, c, 0.0, 0.0])
    np.testing.assert_allclose(Rx @ [0, 1, 0], [0, 0, 1], atol=1e-15)


def test_cov3d_eigenvalues_are_squared_scales():
    rng = np.random.default_rng(5)
    for _ in range(20):
        s = rng.uniform(0.01, 2.0, 3)
        q = rng.standard_normal(4)
        S = oracle.cov3d(s, q)
        np.testing.assert_allclose(S, S.T, atol=1e-14)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(S)), np.sort(s ** 2), rtol=1e-11)


def test_ewa_matches_finite_difference_jacobian():
    """Sigma' - 0.3 I = J Sigma_cam J^T with J the Jacobian of the pinhole map."""
    rng = np.random.default_rng(7)
    cam = scenes.look_at((1.0, 0.5, -5.0), (0.2, -0.1, 0.0), 320, 240, 60.0)
    W = np.asarray(cam["viewmat"], np.float64)[:3, :3]
    fx, fy = float(np.float32(cam["fx"])), float(np.float32(cam["fy"]))

    def proj(t):
        return np.array([fx * t[0] / t[2], fy * t[1] / t[2]])

    for _ in range(10):
        t = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(2.0, 6.0)])
        Sig = oracle.cov3d(rng.uniform(0.01, 0.3, 3), rng.standard_normal(4))
        h = 1e-6
        J = np.stack([(proj(t + h * e) - proj(t - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        ref = J @ W @ Sig @ W.T @ J.T
        got = oracle.ewa(cam, t, Sig)
        np.testing.assert_allclose(got, [ref[0, 0], ref[0, 1], ref[1, 1]], rtol=1e-7, atol=1e-9)
        assert np.all(np.linalg.eigvalsh(ref) >= -1e-12)


def test_ewa_clamps_outside_the_1p3_frustum():
    """Beyond 1.3 tan(fov/2) the Jacobian is taken at the clamped direction."""
    cam = _axis_camera(200, 100, 100.0)
    lim = 1.3 * 200 / (2 * 100.0)
    Sig = np.diag([0.01, 0.02, 0.03])
    t_far = np.array([3.0 * 4.0, 0.1, 4.0])        # x/z = 3 > lim
    t_clamped = np.array([lim * 4.0, 0.1, 4.0])
    np.testing.assert_allclose(oracle.ewa(cam, t_far, Sig), oracle.ewa(cam, t_clamped, Sig),
                               rtol=1e-14)


# --------------------------------------------------------------------------- spherical harmonics
def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi is exact for these polynomials
    xs, ws = np.polynomial.legendre.leggauss(16)
    phis = np.arange(32) * (2 * math.pi / 32)
    idx = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    G = np.zeros((16, 16))
    for x, w in zip(xs, ws):
        st = math.sqrt(1 - x * x)
        for ph in phis:
            d = np.array([st * math.cos(ph), st * math.sin(ph), x])
            y = np.array([oracle.sh_basis(l, m, d) for l, m in idx])
            G += w * (2 * math.pi / 32) * np.outer(y, y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_textbook_values():
    """Closed forms of the real SH (Condon-Shortley phase, Sloan's tables)."""
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        x, y, z = d
        ref = {
            (0, 0): 0.5 * math.sqrt(1 / math.pi),
            (1, -1): -math.sqrt(3 / (4 * math.pi)) * y,
            (1, 0): math.sqrt(3 / (4 * math.pi)) * z,
            (1, 1): -math.sqrt(3 / (4 * math.pi)) * x,
            (2, -2): 0.5 * math.sqrt(15 / math.pi) * x * y,
            (2, -1): -0.5 * math.sqrt(15 / math.pi) * y * z,
            (2, 0): 0.25 * math.sqrt(5 / math.pi) * (3 * z * z - 1),
            (2, 1): -0.5 * math.sqrt(15 / math.pi) * x * z,
            (2, 2): 0.25 * math.sqrt(15 / math.pi) * (x * x - y * y),
            (3, -3): -0.25 * math.sqrt(35 / (2 * math.pi)) * y * (3 * x * x - y * y),
            (3, -2): 0.5 * math.sqrt(105 / math.pi) * x * y * z,
            (3, 0): 0.25 * math.sqrt(7 / math.pi) * (5 * z ** 3 - 3 * z),
            (3, 2): 0.25 * math.sqrt(105 / math.pi) * z * (x * x - y * y),
            (3, 3): -0.25 * math.sqrt(35 / (2 * math.pi)) * x * (x * x - 3 * y * y),
        }
        for (l, m), v in ref.items():
            assert oracle.sh_basis(l, m, d) == pytest.approx(v, abs=1e-13), (l, m)


# --------------------------------------------------------------------------- single Gaussian closed form
@pytest.mark.parametrize("o", [0.3, 0.8, 0.999])
def test_single_gaussian_closed_form(o):
    W = H = 255                                   # odd: the centre pixel (127,127) is the axis
    f, z, s = 200.0, 4.0, 0.02
    dc = 0.7
    cam = _axis_camera(W, H, f)
    sc = _scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[[dc, dc, dc]]])
    r = oracle.render(sc, cam)
    pre = r["pre"]
    o = float(np.float32(o))
    s32 = float(np.float32(s))                    # the oracle consumes float32 inputs
    sig2 = (f * s32 / z) ** 2 + 0.3
    np.testing.assert_allclose(pre["uv"][0], [127.0, 127.0], atol=1e-12)
    np.testing.assert_allclose(pre["conic"][0], [1 / sig2, 0.0, 1 / sig2], rtol=1e-12, atol=1e-15)
    rad = math.ceil(3 * math.sqrt(sig2 + math.sqrt(0.1)))
    assert pre["radius"][0] == rad
    x0, x1 = math.floor((127 - rad) / 16), math.floor((127 + rad + 15) / 16)
    assert list(pre["rect"][0]) == [x0, x0, x1, x1]
    rgb = Y00 * float(np.float32(dc)) + 0.5
    np.testing.assert_allclose(pre["rgb"][0], [rgb] * 3, rtol=1e-14)
    yy, xx = np.mgrid[0:H, 0:W]
    r2 = (xx - 127.0) ** 2 + (yy - 127.0) ** 2
    al = np.minimum(0.99, o * np.exp(-0.5 * r2 / sig2))
    inside = (xx >= 16 * x0) & (xx < 16 * x1) & (yy >= 16 * x0) & (yy < 16 * x1)
    on = (al >= 1 / 255) & inside
    np.testing.assert_allclose(r["rgb"][0], np.where(on, rgb * al, 0.0), atol=1e-14)
    np.testing.assert_allclose(r["final_T"], np.where(on, 1 - al, 1.0), atol=1e-14)
    np.testing.assert_array_equal(r["n_contrib"], on.astype(np.uint32))
    assert r["rgb"][0, 127, 127] == pytest.approx(rgb * min(0.99, o), abs=1e-14)


# --------------------------------------------------------------------------- composition
def test_two_gaussian_composition_front_to_back():
    W = H = 63
    cam = _axis_camera(W, H, 100.0)
    # index 0 is the far one: order must come from depth, not index
    sc = _scene([[0, 0, 6.0], [0, 0, 3.0]], [[0.05] * 3, [0.05] * 3], [[1, 0, 0, 0]] * 2,
                [0.5, 0.6], [[[0.2, 0.4, 0.9]], [[0.8, -0.3, 0.1]]])
    r = oracle.render(sc, cam)
    c_far = Y00 * np.float32([0.2, 0.4, 0.9]).astype(np.float64) + 0.5
    c_near = Y00 * np.float32([0.8, -0.3, 0.1]).astype(np.float64) + 0.5
    a_near, a_far = float(np.float32(0.6)), 0.5                       # the centre pixel sits on both means
    ref = c_near * a_near + c_far * a_far * (1 - a_near)
    np.testing.assert_allclose(r["rgb"][:, 31, 31], ref, rtol=1e-13)
    assert r["final_T"][31, 31] == pytest.approx((1 - a_near) * (1 - a_far), rel=1e-13)
    tile = (31 // 16) * 4 + 31 // 16
    s, e = r["ranges"][tile]
    assert list(r["vals"][s:e]) == [1, 0]


def test_alpha_stack_stops_at_transmittance_threshold():
    W = H = 31
    cam = _axis_camera(W, H, 100.0)
    n = 5
    depths = [2.0 + 0.5 * k for k in range(n)]
    sc = _scene([[0, 0, d] for d in depths], [[0.05] * 3] * n, [[1, 0, 0, 0]] * n, [0.95] * n,
                [[[0.3 * k, 0.1, -0.2]] for k in range(n)])
    r = oracle.render(sc, cam)
    # T: 1 -> 0.05 -> 0.0025 -> 1.25e-4; the 4th would give 6.25e-6 < 1e-4: stop
    assert r["n_contrib"][15, 15] == 3
    assert r["stop_pos"][15, 15] == 4
    assert r["final_T"][15, 15] == pytest.approx(1.25e-4, rel=1e-6)
    cols = [Y00 * np.float32([0.3 * k, 0.1, -0.2]).astype(np.float64) + 0.5 for k in range(3)]
    a = float(np.float32(0.95))
    T = [1.0, 1 - a, (1 - a) ** 2]
    ref = sum(np.maximum(c, 0) * a * t for c, t in zip(cols, T))
    np.testing.assert_allclose(r["rgb"][:, 15, 15], ref, rtol=1e-12)


def test_background_composites_with_final_transmittance():
    cam = _axis_camera(31, 31, 100.0, bg=(0.25, 0.5, 1.0))
    sc = _scene([[0, 0, 3.0]], [[0.05] * 3], [[1, 0, 0, 0]], [0.7], [[[0.0, 0.0, 0.0]]])
    r = oracle.render(sc, cam)
    a = float(np.float32(0.7))
    np.testing.assert_allclose(r["rgb"][:, 15, 15], 0.5 * a + (1 - a) * np.array([0.25, 0.5, 1.0]),
                               rtol=1e-13)
    np.testing.assert_allclose(r["rgb"][:, 0, 0], [0.25, 0.5, 1.0])


# --------------------------------------------------------------------------- invariants
def test_blend_invariants_random_scene():
    sc, cams = scenes.random_small(400, seed=11, width=70, height=45)
    r = oracle.render(sc, cams[0])
    T = r["final_T"]
    assert np.all(T <= 1.0) and np.all(T >= 1e-4)
    pre = r["pre"]
    maxc = pre["rgb"].max()
    assert np.all(r["rgb"] >= 0.0)
    assert np.all(r["rgb"] <= maxc * (1 - T)[None] + 1e-12)
    lens = (r["ranges"][:, 1] - r["ranges"][:, 0])
    gx = (70 + 15) // 16
    tile_of = (np.arange(45)[:, None] // 16) * gx + np.arange(70)[None, :] // 16
    assert np.all(r["n_contrib"] <= lens[tile_of])
    assert np.all(r["n_useful"] <= r["n_contrib"])


def test_sort_matches_bruteforce_emission():
    sc, cams = scenes.random_small(300, seed=12, width=90, height=50)
    cam = cams[0]
    r = oracle.render(sc, cam)
    pre = r["pre"]
    gx = (90 + 15) // 16
    emitted = []
    for i in range(300):
        x0, y0, x1, y1 = pre["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                emitted.append((((ty * gx + tx) << 32) | int(pre["depth_bits"][i]), len(emitted), i))
    emitted.sort()
    assert [e[0] for e in emitted] == [int(k) for k in r["keys"]]
    assert [e[2] for e in emitted] == [int(v) for v in r["vals"]]
    for t in range(r["ranges"].shape[0]):
        s, e = r["ranges"][t]
        sel = [k for k, e_ in enumerate(emitted) if (e_[0] >> 32) == t]
        if sel:
            assert (s, e) == (sel[0], sel[-1] + 1)
        else:
            assert (s, e) == (0, 0)


def _bruteforce(pre, W, H, restrict_to_rect, tile=16):
    """Per pixel over ALL Gaussians sorted by (float32 depth, index): no tiles."""
    n = pre["uv"].shape[0]
    vis = np.nonzero(pre["tiles"] > 0)[0]
    depth32 = pre["depth_bits"].view(np.float32)
    order = vis[np.lexsort((vis, depth32[vis]))]
    img = np.zeros((3, H, W))
    TT = np.ones((H, W))
    for py in range(H):
        for px in range(W):
            T, C = 1.0, np.zeros(3)
            for i in order:
                if restrict_to_rect:
                    x0, y0, x1, y1 = pre["rect"][i]
                    if not (x0 <= px // tile < x1 and y0 <= py // tile < y1):
                        continue
                d = pre["uv"][i] - (px, py)
                a, b, c = pre["conic"][i]
                q = a * d[0] ** 2 + 2 * b * d[0] * d[1] + c * d[1] ** 2
                al = min(0.99, float(pre["opacity"][i]) * math.exp(-0.5 * q))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                C += pre["rgb"][i] * al * T
                T *= 1 - al
            img[:, py, px] = C
            TT[py, px] = T
    assert n >= len(vis)
    return img, TT


def test_bruteforce_without_tiles_low_opacity():
    """With o <= 0.35 every alpha >= 1/255 lies inside the 3-sigma rect, so the
    tiled result must equal a per-pixel loop over all Gaussians without tiles."""
    sc, cams = scenes.random_small(120, seed=21, width=40, height=33, opacity_max=0.35)
    r = oracle.render(sc, cams[0])
    img, TT = _bruteforce(r["pre"], 40, 33, restrict_to_rect=False)
    np.testing.assert_allclose(r["rgb"], img, atol=1e-12)
    np.testing.assert_allclose(r["final_T"], TT, atol=1e-12)


def test_bruteforce_with_rect_predicate_any_opacity():
    sc, cams = scenes.random_small(100, seed=22, width=37, height=29)
    r = oracle.render(sc, cams[0])
    img, TT = _bruteforce(r["pre"], 37, 29, restrict_to_rect=True)
    np.testing.assert_allclose(r["rgb"], img, atol=1e-12)
    np.testing.assert_allclose(r["final_T"], TT, atol=1e-12)


# --------------------------------------------------------------------------- Local-GS pieces
def test_hoist_identity():
    """V . [x'^2, x'y', y'^2, x', y', 1] = ln o - 1/2 x~^T Q x~ (Eq. hoist transform)."""
    rng = np.random.default_rng(31)
    for _ in range(200):
        L = rng.standard_normal((2, 2))
        Q = L @ L.T + 0.05 * np.eye(2)
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.01, 0.99)
        dx, dy = rng.uniform(-40, 40, 2)
        V = oracle.hoist(a, b, c, o, dx, dy)
        xp, yp = rng.uniform(-8, 16, 2)
        B = np.array([xp * xp, xp * yp, yp * yp, xp, yp, 1.0])
        xt = np.array([xp - dx, yp - dy])
        ref = math.log(o) - 0.5 * xt @ Q @ xt
        assert V @ B == pytest.approx(ref, abs=1e-11 * (1 + abs(ref) + a * 1600 + c * 1600))


def _row_hits(a, b, c, tau, x0t, x1t, yt):
    """Does the horizontal line y~ = yt meet the ellipse inside [x0t, x1t]?"""
    disc = b * b * yt * yt - a * (c * yt * yt - tau)
    if disc < 0:
        return False
    lo = (-b * yt - math.sqrt(disc)) / a
    hi = (-b * yt + math.sqrt(disc)) / a
    return hi >= x0t and lo <= x1t


def test_warp_mask_equals_exact_row_intersection():
    """Cases A/B/C give the exact vertical extent of ellipse n strip: a warp bit
    is set iff one of its integer rows meets the ellipse inside the column."""
    rng = np.random.default_rng(41)
    n_checked = 0
    for _ in range(3000):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
        Q = np.linalg.inv(L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2))
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.003, 0.99)
        X0, Y0 = 32, 48
        mux, muy = rng.uniform(X0 - 30, X0 + 46), rng.uniform(Y0 - 30, Y0 + 46)
        m = oracle.warp_mask(a, b, c, o, mux, muy, X0, Y0)
        tau = 2 * math.log(255 * o)
        ref = 0
        if tau > 0:
            for row in range(16):
                if _row_hits(a, b, c, tau, X0 - mux, X0 + 15 - mux, Y0 + row - muy):
                    ref |= 1 << (row // 2)
        # skip configurations whose boundary lies within 1e-9 of a row (ties)
        m_eps = 0
        if tau > 0:
            for row in range(16):
                for e in (-1e-7, 1e-7):
                    if _row_hits(a, b, c, tau, X0 - mux, X0 + 15 - mux, Y0 + row + e - muy):
                        m_eps |= 1 << (row // 2)
        if m_eps != ref:
            continue
        n_checked += 1
        assert m == ref, (a, b, c, o, mux, muy, m, ref)
    assert n_checked > 2900


def test_warp_mask_is_superset_of_contributing_pixels():
    rng = np.random.default_rng(42)
    for _ in range(500):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
        Q = np.linalg.inv(L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2))
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.003, 0.99)
        X0, Y0 = 16, 16
        mux, muy = rng.uniform(0, 48), rng.uniform(0, 48)
        m = oracle.warp_mask(a, b, c, o, mux, muy, X0, Y0)
        yy, xx = np.mgrid[Y0:Y0 + 16, X0:X0 + 16]
        dx, dy = xx - mux, yy - muy
        al = o * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        rows = np.nonzero((al >= 1 / 255 * (1 + 1e-12)).any(axis=1))[0]
        for row in rows:
            assert m & (1 << (row // 2))


# --------------------------------------------------------------------------- printed constants
def test_paper_error_bound_constants():
    """Sec. III-B4 prints 4*4000^2*eps ~ 3.81 and 4*32^2*eps ~ 2.44e-4 (eps = 2^-24)."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "error_bounds.json")))
    eps = 2.0 ** -24
    assert 4 * 4000 ** 2 * eps == pytest.approx(g["E_global"], rel=2e-3)
    assert 4 * 32 ** 2 * eps == pytest.approx(g["E_local"], rel=2e-3)
    # the example: x - mu_x = 0.2 gives a quadratic of 0.04
    assert 0.2 ** 2 == pytest.approx(g["example_quadratic"], rel=1e-12)


def test_fp32_local_frame_error_within_printed_bound():
    """Evaluating (x - mu)^2 expanded in float32 stays within the printed bounds:
    global coordinates near 4000 vs tile-local coordinates in [-16, 32]."""
    rng = np.random.default_rng(51)
    eps = 2.0 ** -24
    mu = rng.uniform(3990, 4000, 10000).astype(np.float32)
    x = np.floor(mu).astype(np.float32)
    f32 = np.float32
    glob = x * x - f32(2) * mu * x + mu * mu
    exact = (x.astype(np.float64) - mu.astype(np.float64)) ** 2
    assert np.max(np.abs(glob.astype(np.float64) - exact)) <= 4 * 4000 ** 2 * eps * 1.01
    T = f32(3984)
    xl, ml = x - T, mu - T
    loc = xl * xl - f32(2) * ml * xl + ml * ml
    assert np.max(np.abs(loc.astype(np.float64) - exact)) <= 4 * 32 ** 2 * eps


# --------------------------------------------------------------------------- near plane
def test_near_plane_cull_at_0p2_inclusive():
    """D3: a Gaussian whose camera-space z is <= 0.2 is culled (radius 0, no
    tiles); one just beyond is kept. The means are given as exact doubles, so z
    = 0.2 reaches the comparison unrounded and '<' in place of '<=' (or another
    constant) fails."""
    cam = _axis_camera(63, 63, 100.0)
    zs = [0.19, 0.2, 0.2 * (1 + 1e-12), 0.21]
    n = len(zs)
    sc = {"means": np.array([[0.0, 0.0, z] for z in zs]), "scales": np.full((n, 3), 1e-3),
          "quats": np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), "opacities": np.full(n, 0.8),
          "sh": np.full((n, 1, 3), 0.3)}
    pre = oracle.preprocess(sc, cam, exact=True)
    np.testing.assert_array_equal(pre["radius"] > 0, [False, False, True, True])
    np.testing.assert_array_equal(pre["tiles"] > 0, [False, False, True, True])
    np.testing.assert_array_equal(pre["depth"], zs)
    # the cull decision at exactly 0.2 lies in the near-plane guard band
    assert pre["gflags"][1] & oracle.GF_NEAR
    assert not pre["gflags"][3] & oracle.GF_NEAR


# --------------------------------------------------------------------------- Local-GS work count
def test_localgs_pairs_single_gaussian_equals_row_intersections():
    """Without a stop, the pair count of one Gaussian is, per tile of its list,
    the number of 16x2 warp strips whose integer rows meet its alpha = 1/255
    ellipse inside the tile column (brute force over rows, as in the warp-mask
    pin), times the 32 pixels of a strip."""
    rng = np.random.default_rng(61)
    cam = _axis_camera(96, 96, 100.0)
    checked = 0
    for trial in range(40):
        z = 4.0
        s = rng.uniform(0.02, 0.12, 3)
        q = rng.standard_normal(4)
        mx, my = rng.uniform(-1.0, 1.0, 2)
        o = rng.uniform(0.05, 0.6)
        sc = _scene([[mx, my, z]], [s], [q], [o], [[[0.2, 0.2, 0.2]]])
        r = oracle.render(sc, cam)
        pre = r["pre"]
        a, b, c = pre["conic"][0]
        ou = float(np.float32(o))
        tau = 2 * math.log(255 * ou)
        mux, muy = pre["uv"][0]
        ref = 0
        ambiguous = False
        gx = 6
        for t in range(gx * gx):
            st, en = r["ranges"][t]
            if en <= st:
                continue
            X0, Y0 = (t % gx) * 16, (t // gx) * 16
            for w in range(8):
                hit = any(_row_hits(a, b, c, tau, X0 - mux, X0 + 15 - mux, Y0 + 2 * w + k - muy)
                          for k in range(2))
                hit_eps = [any(_row_hits(a, b, c, tau, X0 - mux, X0 + 15 - mux, Y0 + 2 * w + k + e - muy)
                               for k in range(2)) for e in (-1e-7, 1e-7)]
                ambiguous |= hit_eps[0] != hit or hit_eps[1] != hit
                ref += 32 * hit
        if ambiguous or tau <= 0:
            continue
        assert r["stop_pos"].max() == 0
        assert oracle.localgs_pairs(r, cam) == ref, trial
        checked += 1
    assert checked >= 30


def test_localgs_pairs_stop_at_the_warps_last_stop_position():
    """A stack of five wide alpha ~ 0.95 Gaussians over a single 16x16 tile:
    every pixel stops at list position 4 (T: 1 -> ~0.05 -> ~2.5e-3 -> ~1.3e-4,
    then T(1 - alpha) < 1e-4), so each of the 8 warps is counted for exactly
    the first 4 Gaussians of the list: 8 x 4 x 32 = 1024 pairs, not the
    5 x 256 = 1280 of the whole list."""
    cam = _axis_camera(16, 16, 100.0)
    n = 5
    depths = [2.0 + 0.5 * k for k in range(n)]
    sc = _scene([[0, 0, d] for d in depths], [[1.0] * 3] * n, [[1, 0, 0, 0]] * n, [0.95] * n,
                [[[0.1 * k, 0.1, 0.1]] for k in range(n)])
    r = oracle.render(sc, cam)
    assert np.all(r["stop_pos"] == 4)
    assert np.all(r["n_contrib"] == 3)
    assert r["ranges"][0][1] - r["ranges"][0][0] == n
    assert oracle.localgs_pairs(r, cam) == 8 * 4 * 32


@pytest.mark.parametrize("block", [(8, 4), (8, 8), (16, 4), (4, 8)])
def test_block_mask_equals_exact_row_intersection_per_block_column(block):
    """2D warp blocks: the bit of block (bx, by) is set iff one of the block's
    integer rows meets the ellipse inside the block's own column range."""
    bw, bh = block
    rng = np.random.default_rng(43 + bw + bh)
    nbx, nby = 16 // bw, 16 // bh
    checked = 0
    for _ in range(1500):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
        Q = np.linalg.inv(L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2))
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.003, 0.99)
        X0, Y0 = 32, 48
        mux, muy = rng.uniform(X0 - 30, X0 + 46), rng.uniform(Y0 - 30, Y0 + 46)
        m = oracle.block_mask(a, b, c, o, mux, muy, X0, Y0, 16, 16, bw, bh)
        tau = 2 * math.log(255 * o)
        refs = []
        for e in (0.0, -1e-7, 1e-7):
            ref = 0
            if tau > 0:
                for bx in range(nbx):
                    x0, x1 = X0 + bx * bw - mux, X0 + bx * bw + bw - 1 - mux
                    for row in range(16):
                        if _row_hits(a, b, c, tau, x0, x1, Y0 + row + e - muy):
                            ref |= 1 << ((row // bh) * nbx + bx)
            refs.append(ref)
        if len(set(refs)) != 1:
            continue
        checked += 1
        assert m == refs[0], (block, a, b, c, o, mux, muy, m, refs[0])
    assert checked > 1400


@pytest.mark.parametrize("block", [(8, 4), (8, 8)])
def test_block_mask_is_superset_of_contributing_pixels(block):
    bw, bh = block
    rng = np.random.default_rng(44)
    nbx = 16 // bw
    for _ in range(400):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
        Q = np.linalg.inv(L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2))
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.003, 0.99)
        X0, Y0 = 16, 16
        mux, muy = rng.uniform(0, 48), rng.uniform(0, 48)
        m = oracle.block_mask(a, b, c, o, mux, muy, X0, Y0, 16, 16, bw, bh)
        yy, xx = np.mgrid[Y0:Y0 + 16, X0:X0 + 16]
        dx, dy = xx - mux, yy - muy
        al = o * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
        for r, cc in zip(*np.nonzero(al >= 1 / 255 * (1 + 1e-12))):
            assert m & (1 << ((r // bh) * nbx + cc // bw))


def test_block_mask_with_full_width_blocks_is_the_strip_mask():
    rng = np.random.default_rng(45)
    for _ in range(300):
        L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
        Q = np.linalg.inv(L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2))
        a, b, c = Q[0, 0], Q[0, 1], Q[1, 1]
        o = rng.uniform(0.003, 0.99)
        mux, muy = rng.uniform(0, 48), rng.uniform(0, 48)
        assert oracle.block_mask(a, b, c, o, mux, muy, 16, 16, 16, 16, 16, 2) == \
            oracle.warp_mask(a, b, c, o, mux, muy, 16, 16)


@pytest.mark.parametrize("block", [(8, 4), (8, 8), (16, 4)])
def test_localgs_pairs_blocks_single_gaussian_and_stack(block):
    """The block count: one Gaussian, no stop -> (blocks whose rows meet its
    ellipse inside their own column range) x block pixels, summed over the
    tiles of its list; the alpha ~ 0.95 stack -> every block counted for the
    first 4 Gaussians: 4 x 256 = 1024 pairs per 16x16 tile, any block shape."""
    bw, bh = block
    nbx = 16 // bw
    rng = np.random.default_rng(62)
    cam = _axis_camera(96, 96, 100.0)
    checked = 0
    for trial in range(30):
        sc = _scene([[*rng.uniform(-1.0, 1.0, 2), 4.0]], [rng.uniform(0.02, 0.12, 3)],
                    [rng.standard_normal(4)], [rng.uniform(0.05, 0.6)], [[[0.2, 0.2, 0.2]]])
        r = oracle.render(sc, cam)
        pre = r["pre"]
        a, b, c = pre["conic"][0]
        tau = 2 * math.log(255 * float(np.float32(sc["opacities"][0])))
        mux, muy = pre["uv"][0]
        ref, ambiguous = 0, False
        for t in range(36):
            st, en = r["ranges"][t]
            if en <= st:
                continue
            X0, Y0 = (t % 6) * 16, (t // 6) * 16
            for w in range(256 // (bw * bh)):
                bx, by = w % nbx, w // nbx
                x0, x1 = X0 + bx * bw - mux, X0 + bx * bw + bw - 1 - mux
                hits = [any(_row_hits(a, b, c, tau, x0, x1, Y0 + by * bh + k + e - muy) for k in range(bh))
                        for e in (0.0, -1e-7, 1e-7)]
                ambiguous |= len(set(hits)) != 1
                ref += bw * bh * hits[0]
        if ambiguous or tau <= 0:
            continue
        assert oracle.localgs_pairs(r, cam, block=block) == ref, trial
        checked += 1
    assert checked >= 20
    cam16 = _axis_camera(16, 16, 100.0)
    n = 5
    st = _scene([[0, 0, 2.0 + 0.5 * k] for k in range(n)], [[1.0] * 3] * n, [[1, 0, 0, 0]] * n,
                [0.95] * n, [[[0.1 * k, 0.1, 0.1]] for k in range(n)])
    assert oracle.localgs_pairs(oracle.render(st, cam16), cam16, block=block) == 4 * 256
