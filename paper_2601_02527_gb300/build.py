"""Build libgpss.so (CUDA for sm_103a) in-tree.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2601_02527_gb300/libgpss.so``.  Run ``python -m paper_2601_02527_gb300.build``
or call :func:`build`.
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
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgpss.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["gpss_api.cu", "gpss_inst_t1.cu", "gpss_inst_t2.cu", "gpss_inst_t2s3.cu",
           "gpss_inst_t2l1.cu", "gpss_inst_i.cu", "gpss_inst_p.cu", "gpss_c64_t1.cu",
           "gpss_c64_t2.cu", "gpss_c64_t3.cu"]


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
            *ARCH, *extra]


def _compile(src: str, extra, objdir=OBJDIR) -> str:
    obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc_path(), "-c", os.path.join(CSRC, src), "-o", obj, *_flags(extra)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "gpss.h"),
                                                               __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), out: str = LIB) -> str:
    """Compile every CUDA translation unit and link libgpss.so (or ``out``,
    with its objects beside it, e.g. a build with extra -D flags); returns
    its path."""
    if out == LIB and not force and not _stale():
        return LIB
    objdir = OBJDIR if out == LIB else os.path.join(os.path.dirname(os.path.abspath(out)),
                                                    "_objs")
    os.makedirs(objdir, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, objdir), SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc_path(), "-shared", "-o", tmp, *objs, *ARCH, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    if verbose:
        print("built", out)
    return out


if __name__ == "__main__":
    extra = sys.argv[1:]
    build(force=True, verbose=True, extra=extra)
