"""Pins of the oracle's hand-derived adjoint against FP64 central finite
differences of the oracle's forward map (CPU only).

L = <g, rgb> + <gT, final_T> with random g, gT. Parameters whose +-h step
changes any piecewise-constant decision (tile rect, radius, alpha >= 1/255
skip, stop position, contributor count) are excluded and counted; the rest
must agree to 1e-5 relative per parameter tensor.
"""
import numpy as np
import pytest

import oracle
from paper_2606_16566_gb300 import scenes

PARAMS = ["means", "scales", "quats", "opacities", "sh"]


def _f64(sc):
    return {k: np.asarray(v, np.float32).astype(np.float64) for k, v in sc.items()}


def _loss(sc, cam, g, gT):
    r = oracle.render(sc, cam, exact=True)
    return float((g * r["rgb"]).sum() + (gT * r["final_T"]).sum()), r


def _signature(r):
    pre = r["pre"]
    return (r["n_contrib"].tobytes(), r["stop_pos"].tobytes(), r["n_useful"].tobytes(),
            pre["tiles"].tobytes(), pre["radius"].tobytes(), pre["rect"].tobytes())


def _fd_check(sc, cam, ids, rel_tol=1e-5, seed=0):
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((3, H, W))
    gT = rng.standard_normal((H, W))
    adj = oracle.backward(sc, cam, g, gT, exact=True)
    _, base = _loss(sc, cam, g, gT)
    sig0 = _signature(base)
    report = {}
    for key in PARAMS:
        fd_all, ad_all, skipped = [], [], 0
        per = int(np.prod(sc[key].shape[1:]))
        for i in ids:
            for e in range(per):
                th = sc[key].reshape(-1)[i * per + e]
                h = 1e-6 * max(1.0, abs(th))
                vals = []
                ok = True
                for sgn in (1.0, -1.0):
                    sc2 = {k: v.copy() for k, v in sc.items()}
                    sc2[key].reshape(-1)[i * per + e] = th + sgn * h
                    Lv, r = _loss(sc2, cam, g, gT)
                    ok &= _signature(r) == sig0
                    vals.append(Lv)
                if not ok:
                    skipped += 1
                    continue
                fd_all.append((vals[0] - vals[1]) / (2 * h))
                ad_all.append(adj[key].reshape(-1)[i * per + e])
        fd_all, ad_all = np.array(fd_all), np.array(ad_all)
        rel = np.linalg.norm(fd_all - ad_all) / max(np.linalg.norm(fd_all), 1e-30)
        report[key] = (rel, skipped, len(fd_all))
        assert rel <= rel_tol, (key, rel, fd_all[:6], ad_all[:6])
    return report, adj


def test_adjoint_matches_fd_sh3():
    sc, cams = scenes.random_small(40, seed=61, width=40, height=32, sh_degree=3, log_scale_mean=-2.3)
    sc = _f64(sc)
    r = oracle.render(sc, cams[0], exact=True)
    vis = np.nonzero(r["pre"]["tiles"] > 0)[0]
    assert len(vis) >= 8
    rep, _ = _fd_check(sc, cams[0], vis[:8])
    print(rep)
    assert sum(n for _, _, n in rep.values()) > 300


def test_adjoint_matches_fd_with_background_and_clamped_alpha():
    """Opacities near 1 make alpha hit the 0.99 clamp at the centre pixels; a
    non-black background exercises the final-T term."""
    sc, cams = scenes.random_small(25, seed=62, width=36, height=30, sh_degree=1, log_scale_mean=-2.0)
    sc = _f64(sc)
    sc["opacities"][:] = np.linspace(0.5, 0.9995, 25)
    cam = dict(cams[0])
    cam["bg"] = np.array([0.2, 0.5, 0.9], np.float32)
    r = oracle.render(sc, cam, exact=True)
    vis = np.nonzero(r["pre"]["tiles"] > 0)[0]
    rep, _ = _fd_check(sc, cam, vis[-6:], seed=1)
    print(rep)


def test_adjoint_near_frustum_clamp():
    """A Gaussian beyond 1.3 tan(fov/2) whose footprint still reaches the image:
    the EWA Jacobian is clamped and its true derivative is used."""
    cam = scenes.look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 48, 40, 60.0)
    n = 6
    sc = {"means": np.array([[1.95, 0.1, 0.0], [2.1, -0.2, 0.3], [0.2, 0.1, 0.0],
                             [-0.3, 0.2, 0.5], [0.1, -0.4, 1.0], [2.4, 0.0, -0.5]], np.float64),
          "scales": np.tile([0.3, 0.12, 0.2], (n, 1)), "quats": np.tile([0.9, 0.1, -0.2, 0.3], (n, 1)),
          "opacities": np.full(n, 0.7), "sh": np.full((n, 4, 3), 0.1)}
    t = (np.asarray(cam["viewmat"], np.float64)[:3, :3] @ sc["means"].T).T + np.asarray(cam["viewmat"], np.float64)[:3, 3]
    lim = 1.3 * 48 / (2 * float(np.float32(cam["fx"])))
    assert np.any(np.abs(t[:, 0] / t[:, 2]) > lim)
    r = oracle.render(sc, cam, exact=True)
    vis = np.nonzero(r["pre"]["tiles"] > 0)[0]
    rep, _ = _fd_check(sc, cam, vis, seed=2)
    print(rep)


def test_adjoint_2d_gradients_consistent():
    """The per-Gaussian 2D gradients dL/d(u, v, a, b, c, o, rgb) agree with
    finite differences through the 3D parameters they feed: dL/do equals the
    3D opacity gradient, and dL/drgb at SH degree 0 is Y00 * dL/dsh."""
    sc, cams = scenes.random_small(30, seed=63, width=32, height=32, sh_degree=0)
    sc = _f64(sc)
    H, W = 32, 32
    g = np.random.default_rng(3).standard_normal((3, H, W))
    adj = oracle.backward(sc, cams[0], g, None, exact=True)
    np.testing.assert_allclose(adj["g2d"][:, 5], adj["opacities"], rtol=1e-12, atol=1e-15)
    Y00 = 0.5 / np.sqrt(np.pi)
    np.testing.assert_allclose(adj["sh"][:, 0, :], Y00 * adj["g2d"][:, 6:9], rtol=1e-12, atol=1e-15)
