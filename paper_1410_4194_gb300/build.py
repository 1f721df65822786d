"""Build the CUDA library ``_build/libhydro.so`` for sm_103a with nvcc.

Translation units compile in parallel; the FP64 kernels are compiled without
fused multiply-add contraction (--fmad=false) so that their arithmetic is the
IEEE sequence the CPU reference performs; the mixed-precision kernels keep FMA.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhydro.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
          "-I" + os.path.join(os.path.dirname(HERE), "include")]
UNITS = {
    "hydro_api.cu": [],
    "hydro_fp64.cu": ["--fmad=false"],      # primitives, update, strict kernels
    "hydro_fp64_fast.cu": ["--fmad=true"],  # fast FP64 stage kernels
    "hydro_noalloc.cu": ["--fmad=false"],   # time step without allocation
    "hydro_mixed.cu": ["--fmad=true"],      # mixed-precision stages
    "hydro_batch.cu": [],                   # batches of grids (host runtime)
    "hydro_selfcheck.cu": [],               # conversion self-check
}


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhydro")
    return exe


def _sources_newer_than(target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    for f in os.listdir(CSRC):
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    hdr = os.path.join(os.path.dirname(HERE), "include", "hydro.h")
    return os.path.getmtime(hdr) > t


def build(force=False, verbose=False):
    """Compile every translation unit and link libhydro.so; returns its path."""
    os.makedirs(OUT, exist_ok=True)
    if not force and not _sources_newer_than(LIB):
        return LIB
    exe = nvcc()

    def compile_one(item):
        src, extra = item
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        cmd = [exe] + ARCH + COMMON + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS.items()))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
