"""Build libvd.so in-tree with nvcc for sm_103a (GB300).

Each .cu file in csrc/ is compiled in parallel to an object, then linked into
paper_1607_00908_gb300/libvd.so; the same sources compiled with -DVD_CHECKED
(index checks before every data-dependent scatter access, include/vd.h) give
libvd_checked.so beside it. Run ``python -m paper_1607_00908_gb300.build``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvd.so")
LIB_CHECKED = os.path.join(HERE, "libvd_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(src: str, extra, tag: str = "") -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + tag + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if r.stderr.strip() and os.environ.get("VD_BUILD_VERBOSE"):
        sys.stderr.write(r.stderr)
    return obj


def _link(objs, lib: str) -> None:
    tmp = lib + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)


def build(verbose: bool = False, extra=(), checked: bool = True) -> str:
    """Compile every CUDA source and link libvd.so (and libvd_checked.so);
    returns the path of libvd.so."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    jobs = [(s, list(extra), "") for s in srcs]
    if checked:
        jobs += [(s, list(extra) + ["-DVD_CHECKED"], "_chk") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 8, len(jobs))) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    _link(objs[: len(srcs)], LIB)
    if checked:
        _link(objs[len(srcs):], LIB_CHECKED)
    if verbose:
        print(f"built {LIB}" + (f" and {LIB_CHECKED}" if checked else ""))
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
