"""Pins of the oracle's tight-box emission rule (Sec. III-C2 tight box used to
drop (Gaussian, tile) instances before the sort), checked against brute force
that shares none of the oracle's case analysis."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_16566_gb300 import scenes

TW, TH = 16, 16


def _random_conic(rng):
    L = rng.standard_normal((2, 2)) * rng.uniform(0.05, 1.0)
    Q = np.linalg.inv(L @ L.T * rng.uniform(1, 80) + 0.3 * np.eye(2))
    return Q[0, 0], Q[0, 1], Q[1, 1]


def _sampled_span(a, b, c, tau, x0t, x1t, n=20001):
    """Lowest / highest y~ of the ellipse a x^2 + 2bxy + c y^2 <= tau over the
    strip x~ in [x0t, x1t], by dense sampling of x~ (plus the strip ends and the
    ellipse's own extreme abscissae) and the quadratic in y~ at each sample."""
    xs = np.concatenate([np.linspace(x0t, x1t, n), [x0t, x1t]])
    det = a * c - b * b
    dy = math.sqrt(a * tau / det)
    xs = np.concatenate([xs, [-b * dy / a, b * dy / a]])
    xs = xs[(xs >= x0t) & (xs <= x1t)]
    disc = (b * xs) ** 2 - c * (a * xs * xs - tau)
    xs, disc = xs[disc >= 0], disc[disc >= 0]
    if len(xs) == 0:
        return None
    r = np.sqrt(disc)
    return float(((-b * xs - r) / c).min()), float(((-b * xs + r) / c).max())


@pytest.mark.parametrize("th", [1, 16])
def test_tight_rows_equal_sampled_span(th):
    """Kept tile rows = the tile rows holding an integer pixel row within the
    widened span (tau' = 1.001 tau + 0.02, +-1/64 px) of the column strip
    (tile height 1 compares pixel rows directly)."""
    rng = np.random.default_rng(71)
    checked = 0
    TH = th
    for _ in range(1500):
        a, b, c = _random_conic(rng)
        o = rng.uniform(0.002, 0.99)
        X0 = 64
        mux, muy = rng.uniform(X0 - 60, X0 + 76), rng.uniform(0, 128)
        ry0, ry1 = 0, 128 // TH
        lo, hi, k, _ = oracle.tight_rows(a, b, c, o, mux, muy, X0, ry0, ry1, tile_h=TH)
        tau = 1.001 * 2 * math.log(255 * o) + 0.02
        ref = set()
        near = False
        if tau > 0:
            sp = _sampled_span(a, b, c, tau, X0 - mux, X0 + TW - 1 - mux)
            if sp is not None:
                ylo, yhi = muy + sp[0] - 1 / 64, muy + sp[1] + 1 / 64
                # sampling and tie cases: skip boundaries within 1e-4 px of an integer
                near = min(abs(ylo - round(ylo)), abs(yhi - round(yhi))) < 1e-4
                for ty in range(ry0, ry1):
                    if max(ty * TH, math.ceil(ylo)) <= min(ty * TH + TH - 1, math.floor(yhi)):
                        ref.add(ty)
            else:
                # strip and ellipse only touch within the sampling resolution
                xr = math.sqrt(c * tau / (a * c - b * b))
                near = min(abs(X0 + TW - 1 - mux + xr), abs(X0 - mux - xr)) < 1e-3
        if near:
            continue
        checked += 1
        got = set(range(lo, hi + 1)) if k else set()
        assert got == ref, (a, b, c, o, mux, muy, got, ref)
    assert checked > 1400


def test_tight_rows_keep_every_contributing_pixel():
    """Every pixel of the rect whose FP64 alpha reaches 1/255 lies in a kept
    tile (the rule is a superset of the contributing region)."""
    rng = np.random.default_rng(72)
    for _ in range(400):
        a, b, c = _random_conic(rng)
        o = rng.uniform(0.002, 0.99)
        mux, muy = rng.uniform(0, 96), rng.uniform(0, 96)
        for tx in range(6):
            lo, hi, k, _ = oracle.tight_rows(a, b, c, o, mux, muy, tx * TW, 0, 6)
            ys, xs = np.mgrid[0:96, tx * TW:tx * TW + TW]
            dx, dy = xs - mux, ys - muy
            al = o * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
            rows = np.unique(ys[al >= 1 / 255] // TH)
            for ty in rows:
                assert k > 0 and lo <= ty <= hi, (a, b, c, o, mux, muy, tx, ty, lo, hi)


def test_tight_rows_guard_marks_boundary_cases():
    """A column strip whose span ends sit right on a tile-row boundary is flagged;
    one far from every boundary is not."""
    a = c = 0.05
    b = 0.0
    o = 0.9
    tau = 1.001 * 2 * math.log(255 * o) + 0.02
    r = math.sqrt(tau / a)
    # upper span end exactly on pixel row 32 (first row of tile row 2)
    muy = 32 - r - 1 / 64
    _, _, _, g1 = oracle.tight_rows(a, b, c, o, 8.0, muy, 0, 0, 8, band_tau=1e-4, band_px=2e-3)
    _, _, _, g2 = oracle.tight_rows(a, b, c, o, 8.0, muy + 0.5 - 16, 0, 0, 8, band_tau=1e-4, band_px=2e-3)
    assert g1 and not g2


def test_tight_emission_is_a_subsequence_and_leaves_the_image_unchanged():
    """Tight-box emission only drops instances whose alpha stays below 1/255 on
    the whole tile: rgb and final_T are bit-identical, every tight tile list is
    a subsequence of the full one, and the last contributor of every pixel is
    the same Gaussian."""
    for seed, tile in ((81, (16, 16)), (82, (8, 32)), (83, (32, 8))):
        sc, cams = scenes.random_small(400, seed=seed, width=150, height=110)
        cam = cams[0]
        tw, th = tile
        full = oracle.render(sc, cam, tw, th)
        tight = oracle.render(sc, cam, tw, th, tight=True)
        assert np.array_equal(full["rgb"], tight["rgb"])
        assert np.array_equal(full["final_T"], tight["final_T"])
        assert len(tight["vals"]) < len(full["vals"])
        assert int(tight["pre"]["tiles"].sum()) == len(full["vals"])
        W, H = cam["width"], cam["height"]
        gx = (W + tw - 1) // tw
        pre = full["pre"]
        for t in range(full["ranges"].shape[0]):
            lf = list(full["vals"][full["ranges"][t][0]:full["ranges"][t][1]])
            lt = list(tight["vals"][tight["ranges"][t][0]:tight["ranges"][t][1]])
            it = iter(lf)
            assert all(x in it for x in lt)                    # subsequence
            ty, tx = divmod(t, gx)
            ys, xs = np.mgrid[ty * th:min(ty * th + th, H), tx * tw:min(tx * tw + tw, W)]
            for gid in set(lf) - set(lt):
                d0, d1 = pre["uv"][gid, 0] - xs, pre["uv"][gid, 1] - ys
                a, b, c = pre["conic"][gid]
                al = pre["opacity"][gid] * np.exp(-0.5 * (a * d0 * d0 + 2 * b * d0 * d1 + c * d1 * d1))
                assert al.max() < 1 / 255
            ncf = full["n_contrib"][ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw]
            nct = tight["n_contrib"][ty * th:(ty + 1) * th, tx * tw:(tx + 1) * tw]
            idf = np.where(ncf > 0, np.asarray(lf + [0], np.int64)[np.maximum(ncf.astype(np.int64) - 1, 0)], -1)
            idt = np.where(nct > 0, np.asarray(lt + [0], np.int64)[np.maximum(nct.astype(np.int64) - 1, 0)], -1)
            assert np.array_equal(idf, idt)
