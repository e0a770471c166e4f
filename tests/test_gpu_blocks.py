"""Warp-block layouts of the Local-GS render (lgs_config.warp_w/warp_h): 2D
blocks whose mask also culls by column (8x4 in 16x16 tiles) and 64-pixel
blocks with two pixels per lane (packed two-wide FP32 arithmetic). A layout
changes only which (warp, Gaussian) pairs are evaluated, never the per-pixel
arithmetic, so every output must equal the paper layout's bit for bit; the
work counted under LGS_FLAG_COUNT is checked against the oracle's count for
the same blocks, and one full outdoor view against the oracle directly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_16566_gb300 import batch, lgs, scenes
from paper_2606_16566_gb300 import _lib as L

from parity import assert_image_parity, full_view_parity, to_numpy_view

pytestmark = pytest.mark.gpu

CASES = [(tile, blk) for tile, blocks in lgs.WARP_BLOCKS.items() for blk in blocks[1:]]


def _frame(g, cams, tile, flags, block=None, batch_size=0):
    cfg = lgs.config(tile, "localgs", flags, batch_size, block)
    n = g["means"].shape[0]
    status = lgs.new_status()
    pre = lgs.preprocess(g, cams, cfg, status=status)
    _, vals, ranges = lgs.sort(pre, n, cams, cfg, max(1 << 16, 8 * n * len(cams)), status=status)
    rgb, T, nc = lgs.render_fwd(pre, vals, ranges, cams, cfg, status=status)
    torch.cuda.synchronize()
    st = lgs.read_status(status)
    assert st[L.ST_CODE] == 0, st
    return rgb, T, nc, st


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("tile,block", CASES)
def test_block_layout_equals_paper_layout(tile, block, tight):
    sc, cams = scenes.random_small(4000, seed=301, width=203, height=151, log_scale_mean=-2.8)
    cams = cams + [scenes.look_at((1.0, 2.0, -4.0), (0, 0, 0), 97, 61, 60.0),
                   scenes.look_at((-2.0, 0.5, -3.5), (0, 0, 0), 130, 121, 50.0, bg=(0.2, 0.5, 0.9))]
    g = lgs.to_device(sc)
    fl = L.FLAG_TIGHT if tight else 0
    ref = _frame(g, cams, tile, fl)
    for nb in (256, 128, 64):
        got = _frame(g, cams, tile, fl, block, nb)
        for a, b in zip(ref[:3], got[:3]):
            torch.testing.assert_close(a, b, rtol=0, atol=0)
    # persistent CTAs pulling tiles from the work queue
    got = _frame(g, cams, tile, fl | L.FLAG_PERSISTENT, block)
    for a, b in zip(ref[:3], got[:3]):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


@pytest.mark.parametrize("tile,block", [((16, 16), (16, 2))] + CASES)
def test_block_pair_count_vs_oracle(tile, block):
    """The GPU block mask is a conservative superset of the exact FP64 one, so
    its pair count is >= the oracle's for the same blocks and within 2 %."""
    sc, cams = scenes.random_small(3000, seed=31, width=200, height=160)
    g = lgs.to_device(sc)
    st = _frame(g, cams, tile, L.FLAG_COUNT, block)[3]
    o = oracle.render(sc, cams[0], tile[0], tile[1])
    ref = oracle.localgs_pairs(o, cams[0], tile[0], tile[1], block=block)
    print(tile, block, int(st[L.ST_PAIRS]), ref)
    assert ref > 0
    assert ref <= st[L.ST_PAIRS] <= 1.02 * ref, (int(st[L.ST_PAIRS]), ref)


def test_2d_blocks_cull_by_column():
    """On the same lists, 8x4 blocks in 16x16 tiles evaluate fewer pairs than the
    16x2 strips (the column-half test drops Gaussians that reach only one half)."""
    sc, cams = scenes.outdoor(n=40000, width=320, height=240, n_views=2)
    g = lgs.to_device(sc)
    strips = _frame(g, cams, (16, 16), L.FLAG_COUNT | L.FLAG_TIGHT)[3][L.ST_PAIRS]
    blocks = _frame(g, cams, (16, 16), L.FLAG_COUNT | L.FLAG_TIGHT, (8, 4))[3][L.ST_PAIRS]
    print("pairs 16x2 strips", int(strips), "8x4 blocks", int(blocks))
    assert blocks < strips


@pytest.mark.parametrize("tile,block", [((8, 32), (8, 8)), ((16, 16), (8, 8))])
def test_outdoor_full_size_view_with_block_layout(tile, block):
    """One full outdoor view (500k Gaussians, 8 views in the batch, tight-box
    emission) in a two-pixels-per-lane layout against the oracle."""
    sc, cams = scenes.outdoor()
    n = sc["means"].shape[0]
    g = lgs.to_device(sc)
    r = batch.Renderer(g, cams, tile=tile, tight=True, block=block)
    r.forward()
    torch.cuda.synchronize()
    r.check()
    vals, ranges = r.lists()
    res = {"rgb": r.images(), "final_T": lgs.split_views(r.T, cams, 0),
           "n_contrib": lgs.split_views(r.nc, cams, 0), "vals": vals, "ranges": ranges}
    view = to_numpy_view(res, 3, cams, n, tile)
    rep, _ = full_view_parity(sc, cams[3], view, tile, tight=True)
    print(rep)
    assert not rep["unexplained_tiles"], rep["unexplained_tiles"][:10]
    assert rep["n_contrib_mismatch"] == 0, rep
    assert_image_parity(rep, "outdoor view 3, block layout")


def test_unsupported_blocks_are_rejected():
    sc, cams = scenes.random_small(200, seed=9)
    g = lgs.to_device(sc)
    res = lgs.render(g, cams)
    for tile, block, mode in (((16, 16), (4, 8), "localgs"), ((8, 32), (16, 4), "localgs"),
                              ((16, 16), (8, 8), "plain"), ((16, 16), (8, 4), "literal")):
        with pytest.raises(L.LgsError) as e:
            lgs.render_fwd(res["pre"], res["vals"], res["ranges"], cams, lgs.config(tile, mode, block=block))
        assert e.value.code == L.LGS_ERR_UNSUPPORTED


def _rel(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("tile,block", CASES)
def test_block_layout_adjoint_matches_oracle(tile, block):
    """The adjoint in a warp-block layout (two pixels per lane for 64-pixel
    blocks) against the oracle's FP64 hand adjoint (<= 1e-3 per tensor), with
    a non-black background and dL/dT, and against the paper layout's adjoint
    (the same sums in another order of float atomics, <= 1e-5)."""
    sc, cams = scenes.random_small(700, seed=73, width=93, height=71, sh_degree=3, log_scale_mean=-2.6)
    cam = dict(cams[0])
    cam["bg"] = np.array([0.3, 0.1, 0.6], np.float32)
    rng = np.random.default_rng(6)
    H, W = cam["height"], cam["width"]
    g_rgb = rng.standard_normal((3, H, W)).astype(np.float32)
    g_T = rng.standard_normal((H, W)).astype(np.float32)
    g = lgs.to_device(sc)
    grads = {}
    for blk in (None, block):
        cfg = lgs.config(tile, "localgs", 0, 0, blk)
        st = lgs.new_status()
        pre = lgs.preprocess(g, [cam], cfg, status=st)
        _, vals, ranges = lgs.sort(pre, 700, [cam], cfg, 1 << 18, status=st)
        rgb, T, nc = lgs.render_fwd(pre, vals, ranges, [cam], cfg, status=st)
        gr = lgs.render_bwd(g, [cam], cfg, pre, vals, ranges, T, nc, torch.from_numpy(g_rgb).cuda().reshape(-1),
                            torch.from_numpy(g_T).cuda().reshape(-1), status=st)
        torch.cuda.synchronize()
        assert lgs.read_status(st)[L.ST_CODE] == 0
        grads[blk] = {k: v.cpu().numpy() for k, v in gr.items()}
    ref = oracle.backward(sc, cam, g_rgb, g_T, tile[0], tile[1])
    for k in ("means", "scales", "quats", "opacities", "sh"):
        r = _rel(grads[block][k], ref[k])
        same = _rel(grads[block][k], grads[None][k])
        print(tile, block, k, r, same)
        assert r <= 1e-3, (k, r)
        assert same <= 1e-5, (k, same)


@pytest.mark.parametrize("tile,block", [((16, 16), (8, 8)), ((8, 32), (8, 8))])
def test_block_layout_persistent_graph_adjoint(tile, block):
    """The persistent adjoint in a block layout, inside a captured graph with
    view groups, equals the one-CTA-per-tile launch up to float-atomic order."""
    sc, _ = scenes.outdoor(n=30000)
    cams = [scenes.look_at((5 * np.cos(a), 1.0, 5 * np.sin(a)), (0, 0, 0), 190 + 10 * i, 150 - 7 * i, 60.0)
            for i, a in enumerate(np.linspace(0, 6, 4))]
    g = lgs.to_device(sc)
    rs = []
    for pers in (False, True):
        r = batch.Renderer(g, cams, tile=tile, backward=True, tight=True, persistent=pers, block=block,
                           max_group_tiles=300)
        r.d_rgb.copy_(torch.linspace(-1, 1, r.d_rgb.numel(), device="cuda"))
        r.capture()
        r.step()
        torch.cuda.synchronize()
        r.check()
        rs.append(r)
    assert len(rs[0].groups) > 1
    for k in ("means", "scales", "quats", "opacities", "sh"):
        d = (rs[0].grads[k] - rs[1].grads[k]).norm() / rs[0].grads[k].norm().clamp_min(1e-30)
        assert d.item() <= 1e-4, k


BIG = [(32, 32), (16, 32), (32, 16)]


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("tile", BIG)
def test_large_tiles_match_oracle(tile, tight):
    """Tiles of more than 256 pixels (sorted as one tile, rendered by one CTA
    per 16x16 region in 8x8 blocks) against the oracle on the same tiles:
    lists, contributor counts and images at the parity bar, ragged sizes,
    several views in one batch."""
    sc, cams = scenes.random_small(5000, seed=311, width=203, height=151, log_scale_mean=-2.8)
    cams = cams + [scenes.look_at((1.0, 2.0, -4.0), (0, 0, 0), 97, 61, 60.0)]
    g = lgs.to_device(sc)
    res = lgs.render(g, cams, tile=tile, flags=L.FLAG_TIGHT if tight else 0)
    for v in range(len(cams)):
        view = to_numpy_view(res, v, cams, 5000, tile)
        rep, _ = full_view_parity(sc, cams[v], view, tile, tight=tight)
        print(tile, tight, v, rep)
        assert not rep["unexplained_tiles"], rep["unexplained_tiles"][:10]
        assert rep["n_contrib_mismatch"] == 0, rep
        assert_image_parity(rep, f"tile {tile} view {v}")


@pytest.mark.parametrize("tile", BIG)
def test_large_tiles_pair_count_and_persistent(tile):
    sc, cams = scenes.random_small(3000, seed=31, width=200, height=160)
    g = lgs.to_device(sc)
    ref = _frame(g, cams, tile, L.FLAG_COUNT)
    st = ref[3]
    o = oracle.render(sc, cams[0], tile[0], tile[1])
    want = oracle.localgs_pairs(o, cams[0], tile[0], tile[1], block=(8, 8))
    print(tile, int(st[L.ST_PAIRS]), want)
    assert want <= st[L.ST_PAIRS] <= 1.02 * want
    got = _frame(g, cams, tile, L.FLAG_PERSISTENT)
    for a, b in zip(ref[:3], got[:3]):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


@pytest.mark.parametrize("tile", BIG)
def test_large_tiles_adjoint_matches_oracle(tile):
    sc, cams = scenes.random_small(700, seed=74, width=93, height=71, sh_degree=3, log_scale_mean=-2.6)
    cam = dict(cams[0])
    cam["bg"] = np.array([0.3, 0.1, 0.6], np.float32)
    rng = np.random.default_rng(7)
    H, W = cam["height"], cam["width"]
    g_rgb = rng.standard_normal((3, H, W)).astype(np.float32)
    g_T = rng.standard_normal((H, W)).astype(np.float32)
    g = lgs.to_device(sc)
    cfg = lgs.config(tile)
    st = lgs.new_status()
    pre = lgs.preprocess(g, [cam], cfg, status=st)
    _, vals, ranges = lgs.sort(pre, 700, [cam], cfg, 1 << 18, status=st)
    rgb, T, nc = lgs.render_fwd(pre, vals, ranges, [cam], cfg, status=st)
    gr = lgs.render_bwd(g, [cam], cfg, pre, vals, ranges, T, nc, torch.from_numpy(g_rgb).cuda().reshape(-1),
                        torch.from_numpy(g_T).cuda().reshape(-1), status=st)
    torch.cuda.synchronize()
    assert lgs.read_status(st)[L.ST_CODE] == 0
    ref = oracle.backward(sc, cam, g_rgb, g_T, tile[0], tile[1])
    for k in ("means", "scales", "quats", "opacities", "sh"):
        r = _rel(gr[k].cpu().numpy(), ref[k])
        print(tile, k, r)
        assert r <= 1e-3, (k, r)


def test_large_tiles_reject_other_modes():
    sc, cams = scenes.random_small(200, seed=9)
    g = lgs.to_device(sc)
    res = lgs.render(g, cams, tile=(32, 32))
    for mode in ("plain", "literal", "global"):
        with pytest.raises(L.LgsError) as e:
            lgs.render_fwd(res["pre"], res["vals"], res["ranges"], cams, lgs.config((32, 32), mode))
        assert e.value.code == L.LGS_ERR_UNSUPPORTED
    with pytest.raises(L.LgsError) as e:
        lgs.render_fwd(res["pre"], res["vals"], res["ranges"], cams, lgs.config((32, 32), block=(8, 4)))
    assert e.value.code == L.LGS_ERR_UNSUPPORTED
