"""Tight-box emission (LGS_FLAG_TIGHT) on the GPU against the oracle's FP64
rule: per-entry tile counts and tile-list membership bit-exact outside the
guard band, images identical to the full-rect emission, renders and
gradients at the parity bar."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_16566_gb300 import batch, lgs, scenes
from paper_2606_16566_gb300 import _lib as L

from parity import (assert_image_parity, compare_preprocess, full_view_parity, gpu_pre_numpy,
                    guard_gaussians, to_numpy_view)

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (8, 32), (32, 8)]
T = L.FLAG_TIGHT


def _render(scene, cams, tile=(16, 16), mode="localgs", flags=0):
    return lgs.render(lgs.to_device(scene), cams, tile=tile, mode=mode, flags=flags)


def _lists(res):
    vals = res["vals"].cpu().numpy().view(np.uint32).astype(np.int64)
    rr = res["ranges"].cpu().numpy().view(np.uint32).astype(np.int64)
    return [vals[s:e] for s, e in rr]


@pytest.mark.parametrize("tile", TILES)
def test_tight_counts_match_oracle(tile):
    """Instances per Gaussian (the tight counts) equal the oracle's FP64 rule
    outside the guard band."""
    n = 3000
    sc, cams = scenes.random_small(n, seed=91, width=220, height=170, sh_degree=3)
    res = _render(sc, cams, tile=tile, flags=T)
    o = oracle.render(sc, cams[0], tile[0], tile[1], tight=True)
    cg = np.bincount(res["vals"].cpu().numpy().view(np.uint32).astype(np.int64), minlength=n)
    co = np.bincount(np.asarray(o["vals"], np.int64), minlength=n)
    guard = guard_gaussians(o["pre"])
    differ = cg != co
    print(tile, "K", res["K"], len(o["vals"]), "differ", int(differ.sum()), "in band", int(guard.sum()))
    assert not np.any(differ & ~guard)
    assert differ.sum() <= max(2, 1e-4 * n)
    assert res["K"] == int(cg.sum()) < int(o["pre"]["tiles"].sum())


@pytest.mark.parametrize("tile", TILES)
def test_tight_lists_are_exact_subsequences(tile):
    """Against the GPU's own full-rect lists: every tight list is the full list
    with the dropped instances removed, and the dropped set is exactly what the
    FP64 rule drops on the GPU's preprocess values, outside the guard band."""
    sc, cams = scenes.random_small(2500, seed=92, width=200, height=150, log_scale_mean=-2.9)
    tw, th = tile
    full = _render(sc, cams, tile=tile)
    tight = _render(sc, cams, tile=tile, flags=T)
    lf, lt = _lists(full), _lists(tight)
    pre = gpu_pre_numpy(tight["pre"], 2500)
    W, H = cams[0]["width"], cams[0]["height"]
    gx = (W + tw - 1) // tw
    n_guard = n_checked = n_differ = 0
    for t, (a_, b_) in enumerate(zip(lf, lt)):
        ty, tx = divmod(t, gx)
        keep_ref, guard = [], set()
        for gid in a_:
            x0, y0, x1, y1 = pre["rect"][gid]
            lo, hi, k, gd = oracle.tight_rows(*pre["conic"][gid], float(pre["opacity"][gid]),
                                              *pre["uv"][gid], tx * tw, int(y0), int(y1), tw, th,
                                              band_tau=1e-4, band_px=2e-3)
            if gd:
                guard.add(int(gid))
            if k and lo <= ty <= hi:
                keep_ref.append(int(gid))
        n_guard += len(guard)
        n_checked += len(a_)
        got = [int(x) for x in b_]
        it = iter(a_.tolist())
        assert all(x in it for x in got), t
        assert [x for x in got if x not in guard] == [x for x in keep_ref if x not in guard], t
        n_differ += len(set(got) ^ set(keep_ref))
    # decisions taken the other way (all inside the band) are rare; the band itself stays narrow
    assert n_differ <= max(2, 1e-4 * n_checked), (n_differ, n_checked)
    assert n_guard <= 1e-2 * n_checked, (n_guard, n_checked)
    assert tight["K"] < full["K"]


@pytest.mark.parametrize("mode", ["localgs", "plain"])
@pytest.mark.parametrize("tile", TILES)
def test_tight_images_equal_full_rect_images(mode, tile):
    """Dropped instances never blend, so rgb and final_T are bit-identical and
    the last contributor of every pixel is the same Gaussian."""
    sc, cams = scenes.outdoor(n=30000, width=240, height=176, n_views=2)
    full = _render(sc, cams, tile=tile, mode=mode)
    tight = _render(sc, cams, tile=tile, mode=mode, flags=T)
    torch.testing.assert_close(tight["rgb_flat"], full["rgb_flat"], rtol=0, atol=0)
    torch.testing.assert_close(tight["T_flat"], full["T_flat"], rtol=0, atol=0)
    vf = full["vals"].cpu().numpy().view(np.uint32).astype(np.int64)
    vt = tight["vals"].cpu().numpy().view(np.uint32).astype(np.int64)
    rf = full["ranges"].cpu().numpy().view(np.uint32).astype(np.int64)
    rt = tight["ranges"].cpu().numpy().view(np.uint32).astype(np.int64)
    tw, th = tile
    toff = 0
    for v, c in enumerate(cams):
        W, H = c["width"], c["height"]
        gx, gy = (W + tw - 1) // tw, (H + th - 1) // th
        ncf = full["n_contrib"][v].cpu().numpy().view(np.uint32).astype(np.int64)
        nct = tight["n_contrib"][v].cpu().numpy().view(np.uint32).astype(np.int64)
        ys, xs = np.mgrid[0:H, 0:W]
        t = toff + (ys // th) * gx + xs // tw
        idf = np.where(ncf > 0, vf[np.maximum(rf[t, 0] + ncf - 1, 0)], -1)
        idt = np.where(nct > 0, vt[np.maximum(rt[t, 0] + nct - 1, 0)], -1)
        assert np.array_equal(idf, idt), v
        toff += gx * gy


@pytest.mark.parametrize("tile", TILES)
def test_tight_render_matches_oracle(tile):
    sc, cams = scenes.random_small(2500, seed=93, width=181, height=133)
    res = _render(sc, cams, tile=tile, flags=T)
    view = to_numpy_view(res, 0, cams, 2500, tile)
    rep, _ = full_view_parity(sc, cams[0], view, tile, tight=True)
    print(tile, rep)
    assert not rep["unexplained_tiles"], rep
    assert rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, f"tight {tile}")


@pytest.mark.parametrize("mode", ["localgs", "plain"])
def test_tight_backward_matches_oracle_adjoint(mode):
    sc, cams = scenes.random_small(600, seed=94, width=90, height=70, sh_degree=3, log_scale_mean=-2.6)
    cam = cams[0]
    rng = np.random.default_rng(6)
    g_rgb = rng.standard_normal((3, cam["height"], cam["width"]))
    g = lgs.to_device(sc)
    res = lgs.render(g, [cam], mode=mode, flags=T)
    d_rgb = torch.from_numpy(g_rgb.astype(np.float32)).cuda().reshape(-1)
    gr = lgs.render_bwd(g, [cam], res["cfg"], res["pre"], res["vals"], res["ranges"], res["T_flat"],
                        res["nc_flat"], d_rgb)
    ref = oracle.backward(sc, cam, g_rgb)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        a = gr[k].cpu().numpy().reshape(-1).astype(np.float64)
        b = ref[k].reshape(-1)
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 1e-3, (k, rel)


def test_tight_outdoor_full_size():
    """Full outdoor workload (500k Gaussians, 8 views of 1264x832): K shrinks,
    images equal the full-rect emission, one view against the oracle."""
    sc, cams = scenes.outdoor()
    n = sc["means"].shape[0]
    g = lgs.to_device(sc)
    full = lgs.render(g, cams)
    tight = lgs.render(g, cams, flags=T)
    print("K full", full["K"], "K tight", tight["K"])
    assert tight["K"] < 0.8 * full["K"]
    torch.testing.assert_close(tight["rgb_flat"], full["rgb_flat"], rtol=0, atol=0)
    view = to_numpy_view(tight, 3, cams, n, (16, 16))
    rep, o = full_view_parity(sc, cams[3], view, (16, 16), tight=True)
    print(rep)
    assert not rep["unexplained_tiles"], rep["unexplained_tiles"][:10]
    assert rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, "outdoor tight view 3")
    gp = gpu_pre_numpy(tight["pre"], n * len(cams))
    gv = {k: x[3 * n:4 * n] for k, x in gp.items()}
    prep = compare_preprocess(gv, o["pre"], guard_gaussians(o["pre"]))
    print(prep)
    assert prep["tiles_mismatch"] == 0 and prep["differ"] <= max(2, 1e-4 * n), prep


def test_tight_batched_graph_equals_full_rect():
    sc, cams = scenes.outdoor(n=40000, width=200, height=150, n_views=4)
    g = lgs.to_device(sc)
    a = batch.Renderer(g, cams, persistent=True, backward=True)
    b = batch.Renderer(g, cams, persistent=True, backward=True, tight=True)
    for r in (a, b):
        r.d_rgb.fill_(1.0 / r.d_rgb.numel())
        r.capture()
        r.step()
    torch.cuda.synchronize()
    a.check()
    b.check()
    assert b.check()[L.ST_NUM_INSTANCES] < a.check()[L.ST_NUM_INSTANCES]
    torch.testing.assert_close(b.rgb, a.rgb, rtol=0, atol=0)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        d = (b.grads[k] - a.grads[k]).norm() / a.grads[k].norm().clamp_min(1e-30)
        assert d.item() <= 1e-5, k


def test_tight_static_sort_equals_workspace_sort():
    sc, cams = scenes.random_small(4000, seed=95, width=300, height=200)
    g = lgs.to_device(sc)
    cfg = lgs.config(flags=T)
    st = lgs.new_status()
    pre = lgs.preprocess(g, cams, cfg, status=st)
    k1, v1, r1 = lgs.sort(pre, 4000, cams, cfg, 1 << 17, status=st)
    s1 = lgs.read_status(st)
    st2 = lgs.new_status()
    k2, v2, r2 = lgs.sort_static(pre, 4000, cams, cfg, 1 << 17, status=st2)
    s2 = lgs.read_status(st2)
    assert s1[L.ST_CODE] == 0 and s2[L.ST_CODE] == 0
    K = int(s1[L.ST_NUM_INSTANCES])
    assert K == int(s2[L.ST_NUM_INSTANCES]) < int(pre.tiles[:4000].sum().item())
    torch.testing.assert_close(v2[:K], v1[:K], rtol=0, atol=0)
    torch.testing.assert_close(k2[:K], k1[:K], rtol=0, atol=0)
    torch.testing.assert_close(r2, r1, rtol=0, atol=0)


@pytest.mark.parametrize("tile", TILES)
def test_emission_records_of_the_preprocess_change_nothing(tile):
    """With the preprocess's 32-B emission records (lgs_pre_out.emit) the tight
    sort gathers one record per entry instead of rect, xy and conic; keys,
    lists, ranges, counts and images are bit-identical either way."""
    sc, _ = scenes.outdoor(n=60000)
    cams = [scenes.look_at((6.0 * np.cos(a), 1.5, 6.0 * np.sin(a)), (0, 0, 0), 640, 416, 60.0)
            for a in (0.3, 2.1, 4.0)]
    g = lgs.to_device(sc)
    n = sc["means"].shape[0]
    cfg = lgs.config(tile, "localgs", T)
    outs = []
    for emit in (True, False):
        st = lgs.new_status()
        pre = lgs.preprocess(g, cams, cfg, out=lgs.PreOut.empty(n * len(cams), emit=emit), status=st)
        assert (pre.emit is not None) == emit
        cap = 4 * n * len(cams)
        keys, vals, ranges = lgs.sort(pre, n, cams, cfg, cap, status=st)
        rgb, T_, nc = lgs.render_fwd(pre, vals, ranges, cams, cfg, status=st)
        s = lgs.read_status(st)
        assert s[L.ST_CODE] == 0
        K = int(s[L.ST_NUM_INSTANCES])
        outs.append((K, keys[:K].clone(), vals[:K].clone(), ranges.clone(), rgb, T_, nc))
    assert outs[0][0] == outs[1][0]
    for a, b in zip(outs[0][1:], outs[1][1:]):
        assert torch.equal(a, b)
