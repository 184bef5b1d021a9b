"""Builds the C-ABI shared library from ``csrc/`` with nvcc for sm_103a.

Two artefacts, both in ``paper_2411_16583_gb300/_lib/``:

* ``libfg.so``     -- the product: CUDA kernels + host runtime, ``-gencode
  arch=compute_103a,code=sm_103a``.
* ``libfg_emu.so`` -- the same sources compiled for the host with ``FG_EMU`` (every
  block of every kernel runs on the CPU, thread by thread between barriers).  It is a
  test fixture for machines without a GPU and is never loaded by the product path.

Object files are compiled in parallel and reused while their sources are unchanged.
"""
from __future__ import annotations

import glob
import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
BUILDDIR = os.path.join(os.path.dirname(HERE), "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# transform lengths compiled into the host-emulation library (small test grids)
EMU_SIZES = (1, 8, 12, 16, 24, 32, 48, 64, 100, 128, 256)


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc):
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _digest(paths, extra):
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(extra).encode())
    return h.hexdigest()[:16]


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(INCLUDE, "fg.h")]


def build_gpu(jobs=None, verbose=False):
    """Compile libfg.so for sm_103a; returns its path."""
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    out = os.path.join(LIBDIR, "libfg.so")
    flags = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-I", CSRC, "-I", INCLUDE] + ARCH
    stamp = _digest(_sources() + _headers(), flags)
    stamp_file = out + ".stamp"
    if os.path.exists(out) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return out
    bdir = os.path.join(BUILDDIR, "gpu")
    os.makedirs(bdir, exist_ok=True)
    hdr = _digest(_headers(), flags)

    def obj(src):
        o = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        key = _digest([src], [hdr])
        kf = o + ".key"
        if os.path.exists(o) and os.path.exists(kf) and open(kf).read() == key:
            return o
        log = _run([nvcc, "-c", src, "-o", o] + flags + (["-Xptxas", "-v"] if verbose else []))
        if verbose:
            print(log)
        with open(kf, "w") as f:
            f.write(key)
        return o

    jobs = jobs or max(1, os.cpu_count() or 1)
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(obj, _sources()))
    cudart = os.path.join(_cuda_home(nvcc), "lib64")
    _run([nvcc, "-shared", "-o", out] + objs + ARCH + ["-L", cudart, "-lcudart", "-ldl"])
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return out


def build_comparator():
    """Compile libfg_cufft.so, the cuFFT-based comparator of the mechanical operator that
    bench.py times beside the fused path (csrc/comparator/, linked with cuFFT; only its
    fgc_* functions are exported).  Returns its path."""
    nvcc = _nvcc()
    os.makedirs(LIBDIR, exist_ok=True)
    out = os.path.join(LIBDIR, "libfg_cufft.so")
    src = os.path.join(CSRC, "comparator", "fg_cufft_cmp.cu")
    flags = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
             "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE, "-shared"] + ARCH
    stamp = _digest([src] + _headers(), flags)
    stamp_file = out + ".stamp"
    if os.path.exists(out) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return out
    lib = os.path.join(_cuda_home(nvcc), "lib64")
    _run([nvcc, src, "-o", out] + flags + ["-L", lib, "-lcufft", "-lcudart"])
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return out


def build_emu(jobs=None):
    """Compile the host-emulation library libfg_emu.so (test fixture); returns its path."""
    nvcc = _nvcc()
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    os.makedirs(LIBDIR, exist_ok=True)
    out = os.path.join(LIBDIR, "libfg_emu.so")
    cuda_inc = os.path.join(_cuda_home(nvcc), "include")
    srcs = [s for s in _sources()
            if not os.path.basename(s).startswith("fg_size_")
            or int(os.path.basename(s)[8:-3]) in EMU_SIZES]
    flags = ["-x", "c++", "-std=c++17", "-O1", "-fPIC", "-DFG_EMU", "-I", CSRC, "-I", INCLUDE,
             "-I", cuda_inc, "-w"]
    stamp = _digest(srcs + _headers(), flags)
    stamp_file = out + ".stamp"
    if os.path.exists(out) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp:
        return out
    bdir = os.path.join(BUILDDIR, "emu")
    os.makedirs(bdir, exist_ok=True)
    hdr = _digest(_headers(), flags)

    def obj(src):
        o = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        key = _digest([src], [hdr])
        kf = o + ".key"
        if os.path.exists(o) and os.path.exists(kf) and open(kf).read() == key:
            return o
        _run([cxx] + flags + ["-c", src, "-o", o])
        with open(kf, "w") as f:
            f.write(key)
        return o

    jobs = jobs or max(1, os.cpu_count() or 1)
    with ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(obj, srcs))
    _run([cxx, "-shared", "-o", out] + objs)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return out


if __name__ == "__main__":
    what = sys.argv[1:] or ["gpu"]
    if "gpu" in what:
        print(build_gpu(verbose="-v" in what))
    if "emu" in what:
        print(build_emu())
