"""Host-side logic that needs no GPU: view grouping of large batches and the
benchmark's record of the render's DRAM traffic."""
import hashlib
import json
import os
import sys

import pytest

from paper_2606_16566_gb300 import batch
from paper_2606_16566_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cam(w, h):
    return {"width": w, "height": h}


def _tiles(c, tile):
    return ((c["width"] + tile[0] - 1) // tile[0]) * ((c["height"] + tile[1] - 1) // tile[1])


@pytest.mark.parametrize("tile", batch.TILE_SHAPES)
@pytest.mark.parametrize("max_tiles", [300, 5000, 1 << 16])
def test_view_groups_cover_the_views_in_order_within_limits(tile, max_tiles):
    cams = [_cam(w, h) for w, h in ((1920, 1080), (800, 800), (1264, 832), (333, 211), (1920, 800),
                                     (64, 48), (1000, 1000), (1500, 900))]
    groups = batch.view_groups(cams, tile, max_tiles)
    assert groups[0][0] == 0 and groups[-1][1] == len(cams)
    for (a0, a1), (b0, b1) in zip(groups, groups[1:]):
        assert a1 == b0 and a0 < a1
    for v0, v1 in groups:
        t = sum(_tiles(c, tile) for c in cams[v0:v1])
        # a group exceeds the limit only when it is a single view that does
        assert t <= max_tiles or v1 - v0 == 1
        assert v1 - v0 <= L.LGS_MAX_VIEWS
        # greedy: the next view would not have fitted
        if v1 < len(cams):
            assert t + _tiles(cams[v1], tile) > max_tiles


def test_view_groups_respect_the_view_limit():
    cams = [_cam(64, 64)] * (2 * L.LGS_MAX_VIEWS + 3)
    groups = batch.view_groups(cams, (16, 16))
    assert [v1 - v0 for v0, v1 in groups] == [L.LGS_MAX_VIEWS, L.LGS_MAX_VIEWS, 3]


def test_the_headline_and_scale_batches_group_as_measured():
    # 8 views of 1264x832 on 8x32 tiles: one group of 32,864 tiles (two tile-id
    # radix passes); 16 views of 1920x1080: two groups of 8 views
    assert batch.view_groups([_cam(1264, 832)] * 8, (8, 32)) == [(0, 8)]
    assert batch.view_groups([_cam(1920, 1080)] * 16, (16, 16)) == [(0, 8), (8, 16)]


def _fake_tree(tmp_path, render_src, record_src):
    csrc = tmp_path / "paper_2606_16566_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "render.cu").write_bytes(render_src)
    (csrc / "common.cuh").write_bytes(b"// common\n")
    h = hashlib.sha256(record_src + b"// common\n").hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps(
        {"render_localgs_8x32_tight": {"traffic_bytes_per_launch": 123456, "source_sha256_prefix": h}}))


def test_traffic_record_is_used_only_for_the_profiled_sources(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    _fake_tree(tmp_path, b"// kernel v1\n", b"// kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("render_localgs_8x32_tight") == 123456
    assert bench.recorded_traffic("render_localgs_16x16_tight") is None
    (tmp_path / "paper_2606_16566_gb300" / "csrc" / "render.cu").write_bytes(b"// kernel v2\n")
    assert bench.recorded_traffic("render_localgs_8x32_tight") is None


def test_preprocess_output_rows_keep_the_abi_alignment():
    """PreOut.rows (a view group's entries) keeps every array's alignment: 16 B
    for the float4 arrays, 8 B for rect, 32 B for the emission records."""
    from paper_2606_16566_gb300 import lgs
    pre = lgs.PreOut.empty(1000, device="cpu")
    for a, b in ((0, 1000), (3, 17), (501, 999)):
        q = pre.rows(a, b)
        st = q.struct()
        assert st.xy % 16 == 0 and st.conic % 16 == 0 and st.rgb % 16 == 0
        assert st.rect % 8 == 0 and st.emit % 32 == 0
        assert q.emit.shape == (b - a, 8)
    assert lgs.PreOut.empty(10, device="cpu", emit=False).struct().emit is None
