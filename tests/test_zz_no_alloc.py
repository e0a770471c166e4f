"""lgs_sort_static: the sort entry point that allocates nothing.

Some callers of this library cannot allocate device memory at all -- a plugin
inside a host engine that owns every device allocation, or a real-time render
loop that must never enter an allocator after start-up -- so they cannot hand
lgs_sort the workspace it needs. lgs_sort_static keeps that scratch in a
static device array of the library instead. These tests call it through the C
ABI and check that its keys, values and tile ranges equal those of lgs_sort
bit for bit (they are integers), on two calls in a row with different inputs,
so that contents the shared array keeps from the first call cannot leak into
the second; and that sizes beyond its stated maximum are refused up front.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_16566_gb300 import _lib as L
from paper_2606_16566_gb300 import lgs, scenes

pytestmark = pytest.mark.gpu


def _sorted_both_ways(scene, cams, capacity):
    g = lgs.to_device(scene)
    cfg = lgs.config()
    n = scene["means"].shape[0]
    st_ref = lgs.new_status()
    pre = lgs.preprocess(g, cams, cfg, status=st_ref)
    k_ref, v_ref, r_ref = lgs.sort(pre, n, cams, cfg, capacity, status=st_ref)
    s_ref = lgs.read_status(st_ref)
    assert s_ref[L.ST_CODE] == 0
    K = int(s_ref[L.ST_NUM_INSTANCES])
    # outputs pre-filled with garbage: everything compared must be written
    keys = torch.full((capacity,), -1, dtype=torch.int64, device="cuda")
    vals = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full_like(r_ref, -1)
    st = lgs.new_status()
    lgs.sort_static(pre, n, cams, cfg, capacity, keys, vals, ranges, status=st)
    s = lgs.read_status(st)
    assert s[L.ST_CODE] == 0 and s[L.ST_NUM_INSTANCES] == K
    return K, (k_ref, v_ref, r_ref), (keys, vals, ranges)


def test_static_sort_equals_workspace_sort_on_two_calls():
    cap = 1 << 19
    first = scenes.random_small(6000, seed=77, width=300, height=220, log_scale_mean=-2.6)
    second = scenes.random_small(2500, seed=78, width=210, height=170)
    second = (second[0], second[1] + [scenes.look_at((1.5, -1.0, -3.0), (0, 0, 0), 120, 90, 55.0)])
    for scene, cams in (first, second):
        K, ref, got = _sorted_both_ways(scene, cams, cap)
        assert 1000 < K <= cap
        torch.testing.assert_close(got[0][:K], ref[0][:K], rtol=0, atol=0)
        torch.testing.assert_close(got[1][:K], ref[1][:K], rtol=0, atol=0)
        torch.testing.assert_close(got[2], ref[2], rtol=0, atol=0)


def test_static_sort_refuses_sizes_beyond_its_maximum():
    scene, cams = scenes.random_small(100, seed=79)
    g = lgs.to_device(scene)
    cfg = lgs.config()
    pre = lgs.preprocess(g, cams, cfg)
    lib = L.load()
    ps = pre.struct()
    carr = lgs.cameras(cams)
    sentinel = 0x5A5A5A5A5A5A5A5A
    buf = torch.full((16,), sentinel, dtype=torch.int64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    too_many = L.SORT_STATIC_MAX_INSTANCES + 1
    assert lib.lgs_sort_static(ctypes.byref(ps), 100, carr, 1, ctypes.byref(cfg), too_many, p, p, p,
                               p, stream) == L.LGS_ERR_UNSUPPORTED
    too_many_entries = L.SORT_STATIC_MAX_ENTRIES + 1
    assert lib.lgs_sort_static(ctypes.byref(ps), too_many_entries, carr, 1, ctypes.byref(cfg), 1024,
                               p, p, p, p, stream) == L.LGS_ERR_UNSUPPORTED
    # a refused call returns before enqueuing anything: the buffer it was
    # handed for keys, values, ranges and status still holds the sentinel
    torch.cuda.synchronize()
    assert np.all(buf.cpu().numpy() == sentinel)
