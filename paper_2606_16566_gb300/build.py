"""Builds liblgs.so, the sm_103a CUDA library behind include/lgs.h.

Each .cu translation unit is compiled in parallel with nvcc for sm_103a only,
then linked into one shared library with the CUDA runtime linked statically
(so the library loads on any host with the driver, next to any PyTorch
build). The output goes to paper_2606_16566_gb300/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblgs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["preprocess.cu", "sort.cu", "render.cu", "backward.cu", "api.cu", "peaks.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblgs")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                   "-I", CSRC, "--expt-relaxed-constexpr", *extra]


CHECKED_DIR = os.path.join(OUT_DIR, "checked")
CHECKED_LIB = os.path.join(CHECKED_DIR, "liblgs.so")


def _compile(src: str, verbose: bool, out_dir: str = OUT_DIR, defines=()) -> str:
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    extra = (["-Xptxas", "-v"] if verbose else []) + [f"-D{d}" for d in defines]
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose:
        print(r.stderr)
    return obj


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lgs.h"),
                                                                  os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds liblgs.so; with checked=True the bounds-checked test build
    (LGS_CHECKED: every checked index that fails records LGS_ERR_INTERNAL and
    skips its access) into _build/checked/."""
    lib, out_dir = (CHECKED_LIB, CHECKED_DIR) if checked else (LIB, OUT_DIR)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    defines = ("LGS_CHECKED",) if checked else ()
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, out_dir, defines), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
