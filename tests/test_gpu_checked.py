"""The bounds-checked test build (LGS_CHECKED): the same parity cases run
through it without a single recorded violation and with results identical to
the regular build; a corrupted tile range is caught and skipped (status
LGS_ERR_INTERNAL, detail 1020) instead of read past the instance list."""
import numpy as np
import pytest
import torch

from paper_2606_16566_gb300 import batch, lgs, scenes
from paper_2606_16566_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    regular = L.load()
    checked = L.load_checked()
    yield regular, checked
    L._LIB = regular


def _use(lib):
    L._LIB = lib


def _run(sc, cams, tile, mode, flags):
    g = lgs.to_device(sc)
    res = lgs.render(g, cams, tile=tile, mode=mode, flags=flags)
    torch.cuda.synchronize()
    return {k: res[k].clone() for k in ("rgb_flat", "T_flat", "nc_flat", "vals", "ranges")}, res


@pytest.mark.parametrize("flags", [0, L.FLAG_TIGHT])
@pytest.mark.parametrize("mode", ["localgs", "plain"])
@pytest.mark.parametrize("tile", [(16, 16), (8, 32), (32, 8)])
def test_checked_build_matches_and_records_nothing(libs, tile, mode, flags):
    regular, checked = libs
    sc, cams = scenes.random_small(3000, seed=111, width=203, height=151)
    cams = cams + [scenes.look_at((1.0, 2.0, -4.0), (0, 0, 0), 97, 61, 60.0)]
    _use(regular)
    a, _ = _run(sc, cams, tile, mode, flags)
    _use(checked)
    b, res = _run(sc, cams, tile, mode, flags)
    st = lgs.read_status(res["status"])
    assert st[L.ST_CODE] == 0, st
    for k in a:
        torch.testing.assert_close(a[k], b[k], rtol=0, atol=0)


def test_checked_build_backward_and_persistent_graph(libs):
    regular, checked = libs
    sc, cams = scenes.outdoor(n=30000, width=200, height=150, n_views=3)
    out = []
    for lib in (regular, checked):
        _use(lib)
        g = lgs.to_device(sc)
        r = batch.Renderer(g, cams, persistent=True, backward=True, tight=True)
        r.d_rgb.fill_(1.0 / r.d_rgb.numel())
        r.capture()
        r.step()
        torch.cuda.synchronize()
        st = r.check()
        assert st[L.ST_CODE] == 0
        out.append((r.rgb.clone(), {k: r.grads[k].clone() for k in ("means", "scales", "sh")}))
    torch.testing.assert_close(out[0][0], out[1][0], rtol=0, atol=0)
    for k in out[0][1]:
        d = (out[0][1][k] - out[1][1][k]).norm() / out[0][1][k].norm().clamp_min(1e-30)
        assert d.item() <= 1e-5, k


def test_checked_build_catches_a_corrupted_tile_range(libs):
    _, checked = libs
    _use(checked)
    sc, cams = scenes.random_small(500, seed=112, width=64, height=48)
    g = lgs.to_device(sc)
    res = lgs.render(g, cams)
    K = res["K"]
    assert K > 0
    # The corrupted range ends 1000 entries past the K sorted instances. The
    # value buffer is extended by 1000 copies of a valid entry index, so even a
    # build without the check would read only allocated, valid records.
    vals = torch.cat([res["vals"], res["vals"][:1].expand(1000)]).contiguous()
    ranges = res["ranges"].clone()
    ranges[0, 0] = 0
    ranges[0, 1] = K + 1000                          # past the sorted instances
    st = lgs.new_status()
    st[L.ST_NUM_INSTANCES] = K                       # the sort's status words
    rgb, T, nc = lgs.render_fwd(res["pre"], vals, ranges, cams, res["cfg"], status=st)
    s = lgs.read_status(st)
    assert s[L.ST_CODE] == L.LGS_ERR_INTERNAL and s[L.ST_DETAIL] == 1020
