"""Build the CUDA library libbisp.so in-tree for sm_103a (nvcc, parallel compiles).

Used by __graft_entry__.build() and by the Python binding when the library is missing.
build(checked=True) makes libbisp_checked.so instead: the same sources with -DBISP_CHECKED
(device bounds checks that record a failed check in a device word, read by bisp_check_word)
and relocatable device code, in its own build folder.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbisp.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libbisp_checked.so")
SOURCES = ["assign.cu", "fft.cu", "measure.cu", "pair.cu", "plan.cu", "noalloc.cu", "fp64.cu", "stats.cu", "model.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(os.path.dirname(HERE), "include")]


def nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _compile(src, verbose, checked=False):
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, src.replace(".cu", ".o"))
    extra = ["-DBISP_CHECKED", "-rdc=true"] if checked else []
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-6000:]}")
    return obj, r.stderr


def build(force=False, verbose=False, checked=False):
    """Compile every .cu for sm_103a and link libbisp.so (libbisp_checked.so with checked=True);
    returns the library path."""
    lib_path = LIB_CHECKED if checked else LIB
    os.makedirs(BUILD_CHECKED if checked else BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    hdrs.append(os.path.join(os.path.dirname(HERE), "include", "bisp.h"))
    if not force and os.path.exists(lib_path):
        t = os.path.getmtime(lib_path)
        if all(os.path.getmtime(p) < t for p in srcs + hdrs):
            return lib_path
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, verbose, checked), SOURCES))
    if verbose:
        for _, log in res:
            sys.stderr.write(log)
    objs = [o for o, _ in res]
    tmp = lib_path + ".tmp"
    # cuFFT serves only the plain FP64 comparison form (precision BISP_FP64)
    libdir = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(shutil.which(nvcc()) or nvcc()))),
                          "lib64")
    cmd = [nvcc(), *ARCH, "-shared", *(["-rdc=true"] if checked else []), "-o", tmp, *objs, "-lcudart", "-lcufft",
           "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
