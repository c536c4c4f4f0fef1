"""Build the CUDA library (liblbm.so) in-tree for sm_103a.

Each .cu file is compiled by nvcc in parallel, then linked into one shared
library exporting the C ABI of include/lbm.h. A content hash of the sources and
flags skips rebuilding when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbm.so")
    return p


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _digest(extra=()) -> str:
    h = hashlib.sha256()
    files = sorted(glob.glob(os.path.join(CSRC, "*")) + [os.path.join(ROOT, "include", "lbm.h")])
    for f in files:
        with open(f, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()


KERNEL_SOURCES = {
    "fd_stage": ["kernels_fd.cu", "fd_common.cuh"],
    "cs_bulk": ["kernels_cs.cu"],
}
SHARED_SOURCES = ["common.cuh", "ptx.cuh", "kernels.h"]


_TOKENS = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\])*"', re.S)


def code_text(src: str) -> str:
    """Source text without comments and with whitespace runs collapsed, so
    that a digest changes with the code only."""
    s = _TOKENS.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", src)
    return re.sub(r"\s+", " ", s).strip()


def kernel_digest(kernel: str, read=None) -> str:
    """Digest of the code of one kernel's sources and the headers it includes
    (identifies the build a profile of that kernel was taken on; comments and
    layout do not count). `read(name)` returns a file's text (default: the
    working tree)."""
    if read is None:
        def read(name):
            with open(os.path.join(CSRC, name), encoding="utf-8") as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel] + SHARED_SOURCES:
        h.update(f.encode())
        h.update(code_text(read(f)).encode())
    return h.hexdigest()[:16]


BOUNDS_DIR = os.path.join(HERE, "_build_bounds")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, bounds: bool = False) -> str:
    """Compile and link liblbm.so; returns its path. bounds=True builds the
    bounds-checked variant (-DLBM_BOUNDS_CHECK) into _build_bounds/ instead."""
    out_dir = BOUNDS_DIR if bounds else OUT_DIR
    lib_path = os.path.join(out_dir, "liblbm.so")
    os.makedirs(out_dir, exist_ok=True)
    extra = (["-Xptxas", "-v"] if ptxas_info else []) + (["-DLBM_BOUNDS_CHECK"] if bounds else [])
    digest = _digest(extra)
    stamp = os.path.join(out_dir, "liblbm.sha256")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == digest:
                return lib_path
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        return obj, r.stderr

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose or ptxas_info:
        for _, err in results:
            if err.strip():
                print(err)
    objs = [o for o, _ in results]
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as fh:
        fh.write(digest)
    return lib_path


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv, bounds="--bounds" in sys.argv))
