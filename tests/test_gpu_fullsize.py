"""Full-size workloads: the indoor training step (2.8M Gaussians) and the
30M-Gaussian scale scene, forward outputs compared with the oracle on a seeded
sample of tiles (every pixel of a sampled tile, oracle blend restricted to
those tiles), plus the indoor gradient check on a 2k-Gaussian crop against the
oracle adjoint and FP64 central finite differences."""
import numpy as np
import pytest
import torch

import oracle
from paper_2606_16566_gb300 import batch, lgs, scenes
from paper_2606_16566_gb300 import _lib as L

from parity import assert_image_parity, full_view_parity, sample_tiles, to_numpy_view

pytestmark = pytest.mark.gpu


def _check_sampled(sc, cams, res, v, frac, seed, tile=(16, 16), tight=False):
    n = sc["means"].shape[0]
    mask = sample_tiles(cams[v], frac, seed, tile)
    view = to_numpy_view(res, v, cams, n, tile)
    rep, _ = full_view_parity(sc, cams[v], view, tile, tile_mask=mask, tight=tight)
    print(v, rep)
    assert not rep["unexplained_tiles"], rep["unexplained_tiles"][:10]
    assert_image_parity(rep, f"view {v}")


@pytest.mark.parametrize("tight,tile,block", [(False, (16, 16), None), (True, (16, 16), None),
                                              (True, (32, 32), (8, 8))])
def test_indoor_training_step(tight, tile, block):
    """Forward + L1 loss against a seeded random target + full adjoint (the
    benchmark's indoor step uses tight-box emission and the autotuner's tile,
    32x32 tiles rendered as 16x16 regions of 8x8 warp blocks on this scene)."""
    sc, cams = scenes.indoor()
    g = lgs.to_device(sc)
    r = batch.Renderer(g, cams, backward=True, tight=tight, tile=tile, block=block)
    r.forward()
    target = torch.rand(r.rgb.shape, generator=torch.Generator(device="cuda").manual_seed(7), device="cuda")
    loss = (r.rgb - target).abs().mean()
    r.d_rgb.copy_(torch.sign(r.rgb - target) / r.rgb.numel())
    r.backward()
    torch.cuda.synchronize()
    st = r.check()
    assert st[2] > (10_000_000 if tile == (16, 16) else 5_000_000) and np.isfinite(loss.item())
    for k in ("means", "scales", "quats", "opacities", "sh"):
        assert torch.isfinite(r.grads[k]).all(), k
        assert r.grads[k].abs().sum().item() > 0, k
    vals, ranges = r.lists()
    res = {"rgb": r.images(), "final_T": lgs.split_views(r.T, cams, 0),
           "n_contrib": lgs.split_views(r.nc, cams, 0), "vals": vals, "ranges": ranges}
    _check_sampled(sc, cams, res, 0, 0.05, seed=11, tight=tight, tile=tile)


def _indoor_crop(n_keep=2000, win=128):
    sc, cams = scenes.indoor()
    cam = cams[0]
    W, H = cam["width"], cam["height"]
    x0, y0 = (W - win) // 2, (H - win) // 2
    pre = oracle.preprocess(sc, cam)
    vis = np.nonzero(pre["tiles"] > 0)[0]
    c = np.array([x0 + win / 2, y0 + win / 2])
    d = np.abs(pre["uv"][vis] - c).max(1)
    keep = np.sort(vis[np.argsort(d)[:n_keep]])
    crop = {k: np.ascontiguousarray(v[keep]) for k, v in sc.items()}
    return crop, scenes.crop_camera(cam, x0, y0, win, win)


def test_indoor_crop_gradients_large_tiles_vs_oracle():
    """The indoor crop's gradients in the benchmark's indoor launch
    configuration (32x32 tiles, 16x16 regions of 8x8 blocks, two pixels per
    lane) against the oracle's FP64 adjoint on the same tiles."""
    sc, cam = _indoor_crop()
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(22)
    g_rgb = rng.standard_normal((3, H, W)).astype(np.float32)
    g = lgs.to_device(sc)
    res = lgs.render(g, [cam], tile=(32, 32), flags=L.FLAG_TIGHT)
    gr = lgs.render_bwd(g, [cam], res["cfg"], res["pre"], res["vals"], res["ranges"], res["T_flat"],
                        res["nc_flat"], torch.from_numpy(g_rgb).cuda().reshape(-1))
    ref = oracle.backward(sc, cam, g_rgb, None, 32, 32)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        got = gr[k].cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(got - ref[k]) / max(np.linalg.norm(ref[k]), 1e-30)
        print(k, rel)
        assert rel <= 1e-3, (k, rel)


def test_indoor_crop_gradients_vs_oracle_and_fd():
    sc, cam = _indoor_crop()
    H, W = cam["height"], cam["width"]
    rng = np.random.default_rng(21)
    target = rng.uniform(0, 1, (3, H, W))
    g = lgs.to_device(sc)
    res = lgs.render(g, [cam])
    img = res["rgb"][0].double().cpu().numpy()
    d_rgb = np.sign(img - target) / img.size
    gr = lgs.render_bwd(g, [cam], res["cfg"], res["pre"], res["vals"], res["ranges"], res["T_flat"],
                        res["nc_flat"], torch.from_numpy(d_rgb.astype(np.float32)).cuda().reshape(-1))
    gg = {k: v.cpu().numpy().astype(np.float64) for k, v in gr.items()}
    sc64 = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in sc.items()}
    ref = oracle.backward(sc64, cam, d_rgb, None, exact=True)
    for k in ("means", "scales", "quats", "opacities", "sh"):
        rel = np.linalg.norm(gg[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-30)
        print(k, rel)
        assert rel <= 1e-3, (k, rel)
    # central finite differences of the FP64 forward on 12 Gaussians x 59 parameters
    vis = np.nonzero(oracle.preprocess(sc64, cam, exact=True)["tiles"] > 0)[0]
    ids = rng.choice(vis, 12, replace=False)

    def L(s):
        o = oracle.render(s, cam, exact=True)
        return float((d_rgb * o["rgb"]).sum()), o

    _, base = L(sc64)
    fd, ad = [], []
    for k in ("means", "scales", "quats", "opacities", "sh"):
        per = int(np.prod(sc64[k].shape[1:]))
        for i in ids:
            for e in range(per):
                th = sc64[k].reshape(-1)[i * per + e]
                h = 1e-6 * max(1.0, abs(th))
                vals, same = [], True
                for sgn in (1, -1):
                    s2 = {kk: vv.copy() for kk, vv in sc64.items()}
                    s2[k].reshape(-1)[i * per + e] = th + sgn * h
                    Lv, o = L(s2)
                    same &= bool(np.array_equal(o["n_contrib"], base["n_contrib"]) and
                                 np.array_equal(o["n_useful"], base["n_useful"]) and
                                 np.array_equal(o["pre"]["tiles"], base["pre"]["tiles"]))
                    vals.append(Lv)
                if same:
                    fd.append((vals[0] - vals[1]) / (2 * h))
                    ad.append(gg[k].reshape(-1)[i * per + e])
    fd, ad = np.array(fd), np.array(ad)
    rel = np.linalg.norm(ad - fd) / np.linalg.norm(fd)
    print("gpu vs fd", rel, len(fd))
    assert len(fd) > 500 and rel <= 1e-3


def test_scale_30M_sampled_view():
    sc, cams = scenes.scale()
    cams = cams[:4]
    g = lgs.to_device(sc)
    r = batch.Renderer(g, cams, persistent=True)
    r.forward()
    torch.cuda.synchronize()
    r.check()
    vals, ranges = r.lists()
    res = {"rgb": r.images(), "final_T": lgs.split_views(r.T, cams, 0),
           "n_contrib": lgs.split_views(r.nc, cams, 0), "vals": vals, "ranges": ranges}
    _check_sampled(sc, cams, res, 1, 0.04, seed=12)


@pytest.mark.parametrize("tile,block,groups", [((16, 16), (8, 8), 2), ((32, 32), (8, 8), 1)])
def test_scale_30M_bench_configuration(tile, block, groups):
    """The benchmark's scale configuration: all 16 views of 1920x1080 in one
    Renderer with tight-box emission (the tight count fused into the last
    entry pass at this size); 16x16 tiles in two view groups of 8, or 32x32
    tiles in one group; two views checked on sampled tiles."""
    sc, cams = scenes.scale()
    g = lgs.to_device(sc)
    r = batch.Renderer(g, cams, tight=True, tile=tile, block=block)
    assert len(r.groups) == groups
    r.forward()
    torch.cuda.synchronize()
    r.check()
    vals, ranges = r.lists()
    res = {"rgb": r.images(), "final_T": lgs.split_views(r.T, cams, 0),
           "n_contrib": lgs.split_views(r.nc, cams, 0), "vals": vals, "ranges": ranges}
    for v, seed in ((5, 13), (12, 14)):
        _check_sampled(sc, cams, res, v, 0.02, seed=seed, tight=True, tile=tile)
