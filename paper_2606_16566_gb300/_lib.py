"""ctypes binding of liblgs.so (include/lgs.h): structures and entry points.

Argument marshalling only. Every step of the rasterization runs in the CUDA
library; if the library is not built this module raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

LGS_OK = 0
LGS_ERR_ARG = 1
LGS_ERR_ALIGN = 2
LGS_ERR_UNSUPPORTED = 3
LGS_ERR_CAPACITY = 4
LGS_ERR_NONFINITE = 5
LGS_ERR_TIMEOUT = 6
LGS_ERR_CUDA = 7
LGS_ERR_INTERNAL = 8

LGS_MAX_VIEWS = 64
SORT_STATIC_MAX_ENTRIES = 1 << 18
SORT_STATIC_MAX_INSTANCES = 1 << 20
SELFTEST_WORKSPACE_BYTES = 256 << 10
LGS_STATUS_WORDS = 8
ST_CODE, ST_DETAIL, ST_NUM_INSTANCES, ST_NONFINITE, ST_PAIRS, ST_QUEUE, ST_QUEUE_BWD, ST_CANDIDATES = range(8)

MODE_LOCALGS = 0
MODE_PLAIN = 1
MODE_LITERAL = 2
MODE_GLOBAL = 3
FLAG_COUNT = 1
FLAG_PERSISTENT = 2
FLAG_TIGHT = 4
FLAG_ONESWEEP = 8
PROBE_FFMA, PROBE_FFMA2, PROBE_EX2 = 0, 1, 2

_vp = ctypes.c_void_p


class lgs_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 16), ("campos", ctypes.c_float * 3),
                ("bg", ctypes.c_float * 3)]


class lgs_gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("means", _vp), ("scales", _vp), ("quats", _vp), ("opacities", _vp), ("sh", _vp)]


class lgs_config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("flags", ctypes.c_int32), ("warp_w", ctypes.c_int32),
                ("warp_h", ctypes.c_int32)]


class lgs_pre_out(ctypes.Structure):
    _fields_ = [("xy", _vp), ("conic", _vp), ("rgb", _vp), ("depth", _vp), ("radius", _vp),
                ("tiles", _vp), ("rect", _vp), ("flags", _vp), ("emit", _vp)]


class lgs_grads(ctypes.Structure):
    _fields_ = [("means", _vp), ("scales", _vp), ("quats", _vp), ("opacities", _vp), ("sh", _vp),
                ("xy2d", _vp), ("conic2d", _vp), ("rgb2d", _vp)]


# Every symbol the header declares, with its signature.
SIGNATURES = {
    "lgs_preprocess": (ctypes.c_int32, [ctypes.POINTER(lgs_gaussians), ctypes.POINTER(lgs_camera),
                                        ctypes.c_int32, ctypes.POINTER(lgs_config),
                                        ctypes.POINTER(lgs_pre_out), _vp, _vp]),
    "lgs_sort_workspace_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    "lgs_sort": (ctypes.c_int32, [ctypes.POINTER(lgs_pre_out), ctypes.c_int64,
                                  ctypes.POINTER(lgs_camera), ctypes.c_int32,
                                  ctypes.POINTER(lgs_config), ctypes.c_int64, _vp, _vp, _vp, _vp,
                                  ctypes.c_size_t, _vp, _vp]),
    "lgs_sort_static": (ctypes.c_int32, [ctypes.POINTER(lgs_pre_out), ctypes.c_int64,
                                         ctypes.POINTER(lgs_camera), ctypes.c_int32,
                                         ctypes.POINTER(lgs_config), ctypes.c_int64, _vp, _vp, _vp,
                                         _vp, _vp]),
    "lgs_render_fwd": (ctypes.c_int32, [ctypes.POINTER(lgs_pre_out), _vp, _vp,
                                        ctypes.POINTER(lgs_camera), ctypes.c_int32,
                                        ctypes.POINTER(lgs_config), _vp, _vp, _vp, _vp, _vp]),
    "lgs_render_bwd": (ctypes.c_int32, [ctypes.POINTER(lgs_gaussians), ctypes.POINTER(lgs_camera),
                                        ctypes.c_int32, ctypes.POINTER(lgs_config),
                                        ctypes.POINTER(lgs_pre_out), _vp, _vp, _vp, _vp, _vp, _vp,
                                        ctypes.POINTER(lgs_grads), _vp, _vp]),
    "lgs_selftest_wait_timeout": (ctypes.c_int32, [ctypes.c_int32, _vp, ctypes.c_size_t, _vp, _vp]),
    "lgs_read_status": (ctypes.c_int32, [_vp, ctypes.POINTER(ctypes.c_int64), _vp]),
    "lgs_get_device_status": (ctypes.c_int32, [_vp, _vp, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int64)]),
    "lgs_peak_probe": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                        ctypes.POINTER(ctypes.c_double), _vp]),
    "lgs_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "lgs_version": (ctypes.c_int32, []),
}

_LIB = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads liblgs.so (building it with nvcc first if asked and needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"liblgs.so is not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def load_checked():
    """The bounds-checked test build (LGS_CHECKED), built on first use, with the
    same signatures; it does not replace the library load() returns."""
    path = _build.build(checked=True)
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


class LgsError(RuntimeError):
    def __init__(self, code, what=""):
        msg = load().lgs_status_string(code).decode()
        super().__init__(f"{what}: lgs status {code} ({msg})")
        self.code = code


def check(code, what=""):
    if code != LGS_OK:
        raise LgsError(code, what)
