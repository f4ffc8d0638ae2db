"""Build the CUDA libraries in-tree (sm_103a):
  paper_2607_28872_b300/libvct.so        the step's C ABI (include/vct.h)
  paper_2607_28872_b300/libvct_peaks.so  FP32/FP64 FMA throughput probe used by bench.py
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libvct.so")
PEAKS_LIB = os.path.join(HERE, "libvct_peaks.so")
SOURCES = ["vct_kernels.cu", "vct_api.cu"]
PEAKS_SOURCES = ["vct_peaks.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler",
                "-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]


def _mtime(files):
    return max(os.path.getmtime(f) for f in files)


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f not in PEAKS_SOURCES]
    return _mtime(files + [os.path.join(INCLUDE, "vct.h")])


def _link(lib, sources, verbose, stamp):
    """Compile and link; the library's mtime is set to `stamp`, the newest source
    time seen when the build started, so a source edited during the build
    makes the library stale for the next build."""
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    procs, objs = [], []
    for s in sources:   # translation units compile in parallel
        o = os.path.join(bdir, s.replace(".cu", ".o"))
        cmd = [NVCC] + FLAGS + ["-c", os.path.join(CSRC, s), "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((subprocess.Popen(cmd), cmd))
        objs.append(o)
    for p, cmd in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
    cmd = [NVCC, "-shared"] + ARCH + ["-o", lib + ".tmp"] + objs + ["-lcudart"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    os.utime(lib, (stamp, stamp))


def build(force=False, verbose=False):
    t = _deps()
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < t:
        _link(LIB, SOURCES, verbose, t)
    peaks_src = [os.path.join(CSRC, s) for s in PEAKS_SOURCES]
    t = _mtime(peaks_src)
    if force or not os.path.exists(PEAKS_LIB) or os.path.getmtime(PEAKS_LIB) < t:
        _link(PEAKS_LIB, PEAKS_SOURCES, verbose, t)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
