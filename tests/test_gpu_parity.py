"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer outputs (radius, tiles, rect, depth key bits, per-tile Gaussian
lists, n_contrib) are bit-exact outside guard items; images meet
max |err| <= 2e-3 with at most 1e-4 of the pixels above 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_16566_gb300 import lgs, scenes
from paper_2606_16566_gb300 import _lib as L

from parity import (assert_image_parity, compare_preprocess, full_view_parity, gpu_pre_numpy,
                    guard_gaussians, to_numpy_view)

pytestmark = pytest.mark.gpu

TILES = [(16, 16), (8, 32), (32, 8)]


def _render(scene, cams, tile=(16, 16), mode="localgs", **kw):
    g = lgs.to_device(scene)
    return lgs.render(g, cams, tile=tile, mode=mode, **kw)


# --------------------------------------------------------------------------- preprocess
@pytest.mark.parametrize("seed,deg", [(1, 0), (2, 1), (3, 2), (4, 3)])
def test_preprocess_matches_oracle(seed, deg):
    sc, cams = scenes.random_small(3000, seed=seed, width=200, height=150, sh_degree=deg)
    res = _render(sc, cams)
    torch.cuda.synchronize()
    g = gpu_pre_numpy(res["pre"], 3000)
    o = oracle.preprocess(sc, cams[0])
    rep = compare_preprocess(g, o, guard_gaussians(o))
    print(rep)
    assert rep["radius_mismatch"] == 0 and rep["tiles_mismatch"] == 0, rep
    assert rep["rect_mismatch"] == 0 and rep["depth_mismatch"] == 0, rep
    assert rep["differ"] <= max(2, 1e-4 * 3000), rep
    assert rep["uv_max_err"] < 1e-6, rep
    assert rep["rgb_max_err"] < 1e-5, rep
    assert rep["conic_max_rel"] < 1e-4, rep


def test_preprocess_frustum_edge_entries_keep_their_rects():
    """Gaussians scattered well beyond the view frustum with large, anisotropic
    footprints: entries whose projected mean lies outside the image but whose
    rect still reaches it must keep exactly the oracle's radius, tiles and
    rect (the preprocess skips the projection only for entries that cannot
    reach the tile grid)."""
    n = 4000
    sc, cams = scenes.random_small(n, seed=21, width=160, height=120, sh_degree=0, extent=4.0,
                                   log_scale_mean=-2.5, log_scale_std=0.8, dist=3.0)
    res = _render(sc, cams)
    torch.cuda.synchronize()
    g = gpu_pre_numpy(res["pre"], n)
    o = oracle.preprocess(sc, cams[0])
    rep = compare_preprocess(g, o, guard_gaussians(o))
    print(rep)
    assert rep["radius_mismatch"] == 0 and rep["tiles_mismatch"] == 0, rep
    assert rep["rect_mismatch"] == 0 and rep["depth_mismatch"] == 0, rep
    # both sides of the test are exercised: entries in front of the near plane
    # whose projected mean lies off the image, kept (rect reaches in) and culled
    c = cams[0]
    V = np.asarray(c["viewmat"], np.float64)
    t = sc["means"].astype(np.float64) @ V[:3, :3].T + V[:3, 3]
    u = c["fx"] * t[:, 0] / t[:, 2] + c["cx"]
    v = c["fy"] * t[:, 1] / t[:, 2] + c["cy"]
    off_image = (t[:, 2] > 0.2) & ((u < 0) | (u >= 160) | (v < 0) | (v >= 120))
    assert int(np.sum(off_image & (o["tiles"] > 0))) >= 200
    assert int(np.sum(off_image & (o["tiles"] == 0))) >= 1000


def test_preprocess_culls_and_counts_nonfinite():
    sc, cams = scenes.random_small(64, seed=5)
    clean = _render(sc, cams)["pre"].tiles.cpu().numpy()
    # a Gaussian that reaches a tile (its SH is read, and so checked, only then)
    k = next(i for i in range(10, 64) if clean[i] > 0)
    sc["means"][3] = [np.nan, 0, 0]
    sc["scales"][7, 1] = np.inf
    sc["means"][9] = [0.0, 0.0, -10.0]        # behind the camera
    sc["sh"][k, 0, 1] = np.nan
    res = _render(sc, cams)
    st = lgs.read_status(res["status"])
    assert st[L.ST_NONFINITE] == 3
    tiles = res["pre"].tiles.cpu().numpy()
    assert tiles[3] == 0 and tiles[7] == 0 and tiles[9] == 0 and tiles[k] == 0
    assert np.isfinite(res["rgb_flat"].cpu().numpy()).all()


# --------------------------------------------------------------------------- sort
def _host_sort_of_gpu_keys(res, cams, n, tile):
    """Stable sort, on the host, of the keys re-emitted from the GPU's own
    preprocess outputs: the GPU sort must match it bit for bit (no guard)."""
    tw, th = tile
    pre = gpu_pre_numpy(res["pre"], n * len(cams))
    keys, vals = [], []
    toff = 0
    for v, c in enumerate(cams):
        gx = (c["width"] + tw - 1) // tw
        for i in range(n):
            m = v * n + i
            if pre["tiles"][m] == 0:
                continue
            x0, y0, x1, y1 = pre["rect"][m]
            for ty in range(y0, y1):
                for tx in range(x0, x1):
                    keys.append(((toff + ty * gx + tx) << 32) | int(pre["depth_bits"][m]))
                    vals.append(m)
        toff += gx * ((c["height"] + th - 1) // th)
    keys = np.array(keys, dtype=np.uint64)
    vals = np.array(vals, dtype=np.uint32)
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order], toff


@pytest.mark.parametrize("tile", TILES)
def test_sort_bitexact_against_host_stable_sort(tile):
    sc, cams = scenes.random_small(800, seed=9, width=170, height=130)
    cams = cams + [scenes.look_at((2.0, 1.0, -3.0), (0, 0, 0), 97, 61, 70.0)]
    res = _render(sc, cams, tile=tile)
    k_ref, v_ref, nt = _host_sort_of_gpu_keys(res, cams, 800, tile)
    assert res["K"] == len(k_ref)
    np.testing.assert_array_equal(res["keys"].cpu().numpy().view(np.uint64), k_ref)
    np.testing.assert_array_equal(res["vals"].cpu().numpy().view(np.uint32), v_ref)
    ranges = res["ranges"].cpu().numpy().view(np.uint32)
    tid = (k_ref >> np.uint64(32)).astype(np.int64)
    for t in range(nt):
        idx = np.nonzero(tid == t)[0]
        if len(idx):
            assert tuple(ranges[t]) == (idx[0], idx[-1] + 1)
        else:
            assert tuple(ranges[t]) == (0, 0)


def test_sort_many_instances_multi_pass():
    """Enough instances (> 50k) for many blocks of every radix pass, entry
    passes and tile-id passes alike, so the look-back chains span many blocks."""
    sc, cams = scenes.random_small(20000, seed=10, width=640, height=480, log_scale_mean=-2.5)
    res = _render(sc, cams)
    k = res["keys"].cpu().numpy().view(np.uint64)
    assert res["K"] > 50000
    assert np.all(k[1:] >= k[:-1])
    k_ref, v_ref, _ = _host_sort_of_gpu_keys(res, cams, 20000, (16, 16))
    np.testing.assert_array_equal(k, k_ref)
    np.testing.assert_array_equal(res["vals"].cpu().numpy().view(np.uint32), v_ref)


@pytest.mark.parametrize("n,W,H", [(6000, 64, 48), (30000, 96, 64)])
def test_sort_large_tile_segments(n, W, H):
    """Large overlapping Gaussians in a small image: single tiles hold several
    thousand instances, so one tile's list spans more than one radix block and
    the depth order inside it must survive the block boundaries."""
    sc, cams = scenes.random_small(n, seed=12, width=W, height=H, log_scale_mean=-1.3,
                                   log_scale_std=0.3)
    res = _render(sc, cams)
    ranges = res["ranges"].cpu().numpy().view(np.uint32).astype(np.int64)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 4096
    k_ref, v_ref, _ = _host_sort_of_gpu_keys(res, cams, n, (16, 16))
    np.testing.assert_array_equal(res["keys"].cpu().numpy().view(np.uint64), k_ref)
    np.testing.assert_array_equal(res["vals"].cpu().numpy().view(np.uint32), v_ref)


@pytest.mark.parametrize("n", [500, 9000])
def test_sort_depth_ties_keep_emission_order(n):
    """All Gaussians at exactly the same camera depth: every key of a tile is
    equal, so each tile list must be in ascending Gaussian order."""
    rng = np.random.default_rng(13)
    cam = scenes.look_at((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), 80, 64, 60.0)
    sc = {"means": np.stack([rng.uniform(-1, 1, n), rng.uniform(-0.8, 0.8, n), np.zeros(n)], 1).astype(np.float32),
          "scales": np.full((n, 3), 0.05 if n < 1000 else 0.3, np.float32),
          "quats": np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
          "opacities": np.full(n, 0.5, np.float32), "sh": np.full((n, 1, 3), 0.2, np.float32)}
    res = _render(sc, [cam])
    k_ref, v_ref, _ = _host_sort_of_gpu_keys(res, [cam], n, (16, 16))
    assert len(np.unique(k_ref & np.uint64(0xFFFFFFFF))) == 1
    np.testing.assert_array_equal(res["keys"].cpu().numpy().view(np.uint64), k_ref)
    np.testing.assert_array_equal(res["vals"].cpu().numpy().view(np.uint32), v_ref)


def test_sort_without_keys_output():
    sc, cams = scenes.random_small(1500, seed=14, width=120, height=90)
    g = lgs.to_device(sc)
    cfg = lgs.config()
    st = lgs.new_status()
    pre = lgs.preprocess(g, cams, cfg, status=st)
    k1, v1, r1 = lgs.sort(pre, 1500, cams, cfg, 1 << 16, status=st)
    K = int(lgs.read_status(st)[L.ST_NUM_INSTANCES])
    vals = torch.empty(1 << 16, dtype=torch.int32, device="cuda")
    ranges = torch.empty_like(r1)
    ws = torch.empty(lgs.sort_workspace_size(1500, 1 << 16), dtype=torch.uint8, device="cuda")
    import ctypes
    ps = pre.struct()
    L.check(L.load().lgs_sort(ctypes.byref(ps), 1500, lgs.cameras(cams), 1, ctypes.byref(cfg), 1 << 16,
                              None, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(ranges.data_ptr()),
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), ctypes.c_void_p(st.data_ptr()),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.testing.assert_close(vals[:K], v1[:K], rtol=0, atol=0)
    torch.testing.assert_close(ranges, r1, rtol=0, atol=0)


def test_capacity_overflow_reports_needed_count():
    sc, cams = scenes.random_small(500, seed=11)
    g = lgs.to_device(sc)
    cfg = lgs.config()
    status = lgs.new_status()
    pre = lgs.preprocess(g, cams, cfg, status=status)
    lgs.sort(pre, 500, cams, cfg, 10, status=status)
    st = lgs.read_status(status)
    assert st[L.ST_CODE] == L.LGS_ERR_CAPACITY
    assert st[L.ST_DETAIL] == st[L.ST_NUM_INSTANCES] > 10
    assert lgs.get_device_status(status) == (L.LGS_ERR_CAPACITY, int(st[L.ST_DETAIL]))
    assert lgs.get_device_status(lgs.new_status()) == (0, 0)
    res = _render(sc, cams)                       # the retry path sizes itself
    assert res["K"] == st[L.ST_DETAIL]


# --------------------------------------------------------------------------- render
@pytest.mark.parametrize("mode", ["localgs", "plain"])
@pytest.mark.parametrize("tile", TILES)
def test_render_matches_oracle_small(mode, tile):
    sc, cams = scenes.random_small(2500, seed=21, width=181, height=133)
    res = _render(sc, cams, tile=tile, mode=mode)
    view = to_numpy_view(res, 0, cams, 2500, tile)
    rep, _ = full_view_parity(sc, cams[0], view, tile)
    print(mode, tile, rep)
    assert not rep["unexplained_tiles"], rep
    assert rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, f"{mode} {tile}")


def test_render_tiny_config_matches_oracle():
    sc, cams = scenes.tiny()
    res = _render(sc, cams)
    view = to_numpy_view(res, 0, cams, sc["means"].shape[0], (16, 16))
    rep, _ = full_view_parity(sc, cams[0], view, (16, 16))
    print(rep)
    assert not rep["unexplained_tiles"] and rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, "tiny")


def test_multiview_batch_equals_single_views():
    sc, cams = scenes.outdoor(n=20000, width=160, height=104, n_views=3)
    cams = cams + [scenes.look_at((0.5, 3.0, 5.0), (0, 0, 0), 121, 77, 50.0)]
    res = _render(sc, cams)
    for v in range(len(cams)):
        one = _render(sc, [cams[v]])
        torch.testing.assert_close(res["rgb"][v], one["rgb"][0], rtol=0, atol=0)
        torch.testing.assert_close(res["n_contrib"][v], one["n_contrib"][0], rtol=0, atol=0)


def test_localgs_equals_plain_integer_outputs():
    sc, cams = scenes.random_small(4000, seed=23, width=256, height=200, log_scale_mean=-2.8)
    a = _render(sc, cams, mode="localgs")
    b = _render(sc, cams, mode="plain")
    na, nb = a["n_contrib"][0].cpu().numpy(), b["n_contrib"][0].cpu().numpy()
    assert np.mean(na != nb) <= 1e-3
    err = (a["rgb"][0] - b["rgb"][0]).abs().max().item()
    assert err <= 2e-3


def test_empty_and_degenerate_inputs():
    sc, cams = scenes.random_small(10, seed=3)
    empty = {k: v[:0] for k, v in sc.items()}
    res = _render(empty, cams)
    assert res["K"] == 0
    bg = torch.tensor(cams[0]["bg"]).cuda()
    assert torch.allclose(res["rgb"][0], bg[:, None, None].expand_as(res["rgb"][0]))
    assert torch.all(res["final_T"][0] == 1)
    # everything behind the camera
    sc["means"][:, 2] = -10.0
    res = _render(sc, cams)
    assert res["K"] == 0
    # 1x1 image and an image narrower than a tile
    for W, H in [(1, 1), (5, 37)]:
        sc2, cams2 = scenes.random_small(300, seed=4, width=W, height=H)
        r = _render(sc2, cams2)
        view = to_numpy_view(r, 0, cams2, 300, (16, 16))
        rep, _ = full_view_parity(sc2, cams2[0], view, (16, 16))
        assert rep["n_unexplained"] == 0 and rep["max_abs"] <= 2e-3, rep


def test_schedule_pair_count_vs_oracle():
    """LGS_FLAG_COUNT counts the pixel-Gaussian pairs of the Local-GS schedule
    (mask bit set, up to the warp's exit). The GPU mask is a conservative
    superset of the exact FP64 mask, so the count is >= the oracle's and
    within 2% of it."""
    sc, cams = scenes.random_small(3000, seed=31, width=200, height=160)
    res = _render(sc, cams, flags=L.FLAG_COUNT)
    gpu_pairs = lgs.read_status(res["status"])[L.ST_PAIRS]
    o = oracle.render(sc, cams[0])
    ref = oracle.localgs_pairs(o, cams[0])
    assert ref > 0
    assert ref <= gpu_pairs <= 1.02 * ref, (gpu_pairs, ref)


@pytest.mark.parametrize("tile,tight", [((16, 16), False), ((8, 32), True)])
@pytest.mark.parametrize("v", [0, 5])
def test_outdoor_full_size_views(v, tile, tight):
    """Full outdoor workload (500k Gaussians, 8 views of 1264x832 in one batch);
    two views checked in full, on 16x16 tiles with full-rect emission and in
    the benchmark's headline launch configuration (8x32 tiles, tight-box
    emission, one CTA per tile, 256-Gaussian staging batch)."""
    sc, cams = scenes.outdoor()
    n = sc["means"].shape[0]
    res = _render(sc, cams, tile=tile, flags=L.FLAG_TIGHT if tight else 0)
    view = to_numpy_view(res, v, cams, n, tile)
    rep, o = full_view_parity(sc, cams[v], view, tile, tight=tight)
    print(rep)
    assert not rep["unexplained_tiles"], rep["unexplained_tiles"][:10]
    assert rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, f"outdoor view {v}")
    # preprocess of the same view, all 500k Gaussians
    g = gpu_pre_numpy(res["pre"], n * len(cams))
    gv = {k: x[v * n:(v + 1) * n] for k, x in g.items()}
    prep = compare_preprocess(gv, o["pre"], guard_gaussians(o["pre"]))
    print(prep)
    assert prep["radius_mismatch"] == 0 and prep["tiles_mismatch"] == 0, prep
    assert prep["rect_mismatch"] == 0 and prep["depth_mismatch"] == 0, prep
    assert prep["differ"] <= max(2, 1e-4 * n), prep


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("tile", TILES)
def test_reduce_then_scan_equals_onesweep(tile, tight):
    """The default radix passes (reduce-then-scan: upsweep, scan, downsweep) and
    the single-kernel onesweep passes (LGS_FLAG_ONESWEEP) give identical keys,
    values and tile ranges, on a multi-view batch whose entry and tile-id
    passes both span many blocks."""
    sc, cams = scenes.random_small(20000, seed=14, width=480, height=352, log_scale_mean=-2.5)
    cams = cams + [scenes.look_at((2.0, 1.0, -4.0), (0, 0, 0), 333, 215, 55.0)]
    g = lgs.to_device(sc)
    out = []
    for extra in (0, L.FLAG_ONESWEEP):
        cfg = lgs.config(tile, "localgs", (L.FLAG_TIGHT if tight else 0) | extra)
        st = lgs.new_status()
        pre = lgs.preprocess(g, cams, cfg, status=st)
        keys, vals, ranges = lgs.sort(pre, 20000, cams, cfg, 1 << 21, status=st)
        s = lgs.read_status(st)
        assert s[L.ST_CODE] == 0
        K = int(s[L.ST_NUM_INSTANCES])
        assert K > 100000
        out.append((keys[:K].clone(), vals[:K].clone(), ranges.clone()))
    for a, b in zip(*out):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
