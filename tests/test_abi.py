"""The C-ABI library builds, loads and exports every symbol include/lgs.h
declares; host-side argument checks return errors before touching a GPU."""
import ctypes
import os
import re

from paper_2606_16566_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lgs_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = L.load()
    declared = _declared()
    assert {"lgs_preprocess", "lgs_sort", "lgs_render_fwd", "lgs_render_bwd"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(L.SIGNATURES) >= declared


def test_status_strings_and_version():
    lib = L.load()
    assert lib.lgs_version() >= 1
    for code in range(9):
        assert lib.lgs_status_string(code)
    assert b"capacity" in lib.lgs_status_string(L.LGS_ERR_CAPACITY)


def test_host_side_argument_checks_need_no_gpu():
    lib = L.load()
    cam = (L.lgs_camera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 64, 48, 50.0, 50.0
    cfg = L.lgs_config(16, 16, 0, 0, 0)
    pre = L.lgs_pre_out()
    g = L.lgs_gaussians()
    # NULL output structure pointers -> LGS_ERR_ARG before any launch
    assert lib.lgs_preprocess(ctypes.byref(g), cam, 1, ctypes.byref(cfg), None, None, None) == L.LGS_ERR_ARG
    # unsupported tile shape
    bad = L.lgs_config(12, 12, 0, 0, 0)
    fake = ctypes.c_void_p(16)
    pre2 = L.lgs_pre_out(*([16] * 8))
    assert lib.lgs_render_fwd(ctypes.byref(pre2), fake, fake, cam, 1, ctypes.byref(bad), fake, fake,
                              fake, fake, None) == L.LGS_ERR_UNSUPPORTED
    # too many views
    assert lib.lgs_render_fwd(ctypes.byref(pre2), fake, fake, cam, 65, ctypes.byref(cfg), fake,
                              fake, fake, fake, None) == L.LGS_ERR_UNSUPPORTED
    # misaligned float4 array
    pre3 = L.lgs_pre_out(*([16] * 8))
    pre3.xy = 20
    assert lib.lgs_render_fwd(ctypes.byref(pre3), fake, fake, cam, 1, ctypes.byref(cfg), fake,
                              fake, fake, fake, None) == L.LGS_ERR_ALIGN
    # workspace too small for the sort
    assert lib.lgs_sort(ctypes.byref(pre2), 10, cam, 1, ctypes.byref(cfg), 100, fake, fake, fake,
                        fake, 1, fake, None) == L.LGS_ERR_ARG
    assert lib.lgs_sort_workspace_size(10, 100) > 0
    assert pre.xy is None


def test_peak_probe_argument_checks_need_no_gpu():
    lib = L.load()
    ops = ctypes.c_double(0.0)
    fake = ctypes.c_void_p(256)
    assert lib.lgs_peak_probe(L.PROBE_FFMA, 0, 10, fake, ctypes.byref(ops), None) == L.LGS_ERR_ARG
    assert lib.lgs_peak_probe(L.PROBE_FFMA, 4, 10, None, ctypes.byref(ops), None) == L.LGS_ERR_ARG
    assert lib.lgs_peak_probe(L.PROBE_EX2, 4, 0, fake, ctypes.byref(ops), None) == L.LGS_ERR_ARG
    assert lib.lgs_peak_probe(9, 4, 10, fake, ctypes.byref(ops), None) == L.LGS_ERR_UNSUPPORTED
    assert ops.value == 0.0


def test_selftest_argument_checks_need_no_gpu():
    lib = L.load()
    assert lib.lgs_selftest_wait_timeout(10, None, 0, None, None) == L.LGS_ERR_ARG
    fake = ctypes.c_void_p(256)
    assert lib.lgs_selftest_wait_timeout(10, fake, 1024, fake, None) == L.LGS_ERR_ARG
    assert lib.lgs_selftest_wait_timeout(-1, fake, L.SELFTEST_WORKSPACE_BYTES, fake, None) == L.LGS_ERR_ARG
    assert lib.lgs_selftest_wait_timeout(10, ctypes.c_void_p(260), L.SELFTEST_WORKSPACE_BYTES, fake,
                                         None) == L.LGS_ERR_ALIGN


def _header_defines():
    src = open(os.path.join(ROOT, "include", "lgs.h")).read()
    out = {}
    for name, expr in re.findall(r"#define\s+(LGS_\w+)\s+([^/\n]+)", src):
        expr = re.sub(r"(\d+)(?:ull|ll|u)\b", r"\1", expr.strip())
        try:
            out[name] = int(eval(expr, {}))
        except Exception:
            pass
    return out


def test_python_constants_match_the_header():
    d = _header_defines()
    pairs = {"LGS_ERR_ARG": L.LGS_ERR_ARG, "LGS_ERR_ALIGN": L.LGS_ERR_ALIGN,
             "LGS_ERR_UNSUPPORTED": L.LGS_ERR_UNSUPPORTED, "LGS_ERR_CAPACITY": L.LGS_ERR_CAPACITY,
             "LGS_ERR_TIMEOUT": L.LGS_ERR_TIMEOUT, "LGS_ERR_CUDA": L.LGS_ERR_CUDA,
             "LGS_ERR_INTERNAL": L.LGS_ERR_INTERNAL, "LGS_MAX_VIEWS": L.LGS_MAX_VIEWS,
             "LGS_SORT_STATIC_MAX_ENTRIES": L.SORT_STATIC_MAX_ENTRIES,
             "LGS_SORT_STATIC_MAX_INSTANCES": L.SORT_STATIC_MAX_INSTANCES,
             "LGS_SELFTEST_WORKSPACE_BYTES": L.SELFTEST_WORKSPACE_BYTES,
             "LGS_STATUS_WORDS": L.LGS_STATUS_WORDS, "LGS_MODE_LOCALGS": L.MODE_LOCALGS,
             "LGS_MODE_PLAIN": L.MODE_PLAIN, "LGS_MODE_LITERAL": L.MODE_LITERAL,
             "LGS_MODE_GLOBAL": L.MODE_GLOBAL, "LGS_FLAG_COUNT": L.FLAG_COUNT,
             "LGS_FLAG_PERSISTENT": L.FLAG_PERSISTENT, "LGS_FLAG_TIGHT": L.FLAG_TIGHT,
             "LGS_FLAG_ONESWEEP": L.FLAG_ONESWEEP,
             "LGS_ST_NUM_INSTANCES": L.ST_NUM_INSTANCES, "LGS_ST_PAIRS": L.ST_PAIRS,
             "LGS_ST_CANDIDATES": L.ST_CANDIDATES, "LGS_PROBE_FFMA": L.PROBE_FFMA,
             "LGS_PROBE_FFMA2": L.PROBE_FFMA2, "LGS_PROBE_EX2": L.PROBE_EX2}
    for name, val in pairs.items():
        assert d[name] == val, name


def test_unsupported_staging_batch_is_a_host_error():
    lib = L.load()
    cam = (L.lgs_camera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 64, 48, 50.0, 50.0
    fake = ctypes.c_void_p(16)
    pre = L.lgs_pre_out(*([16] * 8))
    for batch in (96, 32, 512, -1):
        cfg = L.lgs_config(16, 16, 0, batch, 0)   # tile_w, tile_h, mode, batch, flags
        assert lib.lgs_render_fwd(ctypes.byref(pre), fake, fake, cam, 1, ctypes.byref(cfg), fake, fake,
                                  fake, fake, None) == L.LGS_ERR_UNSUPPORTED, batch


def test_misaligned_emission_records_are_a_host_error():
    lib = L.load()
    cam = (L.lgs_camera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 64, 48, 50.0, 50.0
    cfg = L.lgs_config(16, 16, 0, 0, 0)
    fake = ctypes.c_void_p(32)
    pre = L.lgs_pre_out(*([32] * 8), 48)          # 16-B but not 32-B aligned
    assert lib.lgs_render_fwd(ctypes.byref(pre), fake, fake, cam, 1, ctypes.byref(cfg), fake, fake,
                              fake, fake, None) == L.LGS_ERR_ALIGN


def test_device_status_query_checks_its_arguments():
    lib = L.load()
    code = ctypes.c_int32(7)
    assert lib.lgs_get_device_status(None, None, ctypes.byref(code), None) == L.LGS_ERR_ARG
    assert code.value == 7


def test_misaligned_parameter_gradients_are_a_host_error():
    # the preprocess adjoint adds to quats and (SH degree 1 and 3) SH
    # gradients 16 B at a time: misaligned rows return before any launch
    lib = L.load()
    cam = (L.lgs_camera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 64, 48, 50.0, 50.0
    cfg = L.lgs_config(16, 16, 0, 0, 0)
    fake = ctypes.c_void_p(256)
    pre = L.lgs_pre_out(*([256] * 8))
    for deg, bad in ((3, "quats"), (3, "sh"), (1, "sh")):
        g = L.lgs_gaussians(10, deg, 256, 256, 256, 256, 256)
        gr = L.lgs_grads(*([256] * 8))
        setattr(gr, bad, 260)
        assert lib.lgs_render_bwd(ctypes.byref(g), cam, 1, ctypes.byref(cfg), ctypes.byref(pre), fake, fake,
                                  fake, fake, fake, None, ctypes.byref(gr), fake, None) == L.LGS_ERR_ALIGN


def test_unsupported_warp_blocks_are_host_errors():
    # the warp-block check runs on the host before any launch, for the forward
    # and the adjoint: blocks outside the supported set, and other than 8x8 for
    # the large (split) tiles, return LGS_ERR_UNSUPPORTED
    lib = L.load()
    cam = (L.lgs_camera * 1)()
    cam[0].width, cam[0].height, cam[0].fx, cam[0].fy = 64, 48, 50.0, 50.0
    fake = ctypes.c_void_p(256)
    pre = L.lgs_pre_out(*([256] * 8))
    g = L.lgs_gaussians(10, 3, 256, 256, 256, 256, 256)
    gr = L.lgs_grads(*([256] * 8))
    for tile, block in (((16, 16), (4, 8)), ((16, 16), (8, 16)), ((8, 32), (16, 4)), ((32, 32), (16, 4)),
                        ((32, 16), (16, 2)), ((32, 8), (16, 4))):
        cfg = L.lgs_config(tile[0], tile[1], 0, 0, 0, block[0], block[1])
        assert lib.lgs_render_fwd(ctypes.byref(pre), fake, fake, cam, 1, ctypes.byref(cfg), fake, fake, fake,
                                  fake, None) == L.LGS_ERR_UNSUPPORTED, (tile, block)
        assert lib.lgs_render_bwd(ctypes.byref(g), cam, 1, ctypes.byref(cfg), ctypes.byref(pre), fake, fake, fake,
                                  fake, fake, None, ctypes.byref(gr), fake, None) == L.LGS_ERR_UNSUPPORTED, (tile, block)
