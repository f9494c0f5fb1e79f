"""Builds the CUDA library ``_build/liblbm_gb300.so`` in-tree for sm_103a (GB300).

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc, then linked into one
shared library with the CUDA runtime linked statically, so the library has no run-time
dependency beyond the driver.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblbm_gb300.so")
# the bounds-checked variant (-DLBM_DEBUG): every kernel access range-checked, out-of-range
# accesses skipped and reported as LBM_ERR_STATE at the next synchronising call
DEBUG_OUT_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_OUT_DIR, "liblbm_gb300_debug.so")
# a variant with 8 x 4 x 2 bricks in place of 4 x 4 x 4 (periodic extents: multiples of 8, 4, 2)
B842_OUT_DIR = os.path.join(HERE, "_build_b842")
B842_LIB = os.path.join(B842_OUT_DIR, "liblbm_gb300_b842.so")
B842_FLAGS = ("-DLBM_BRICK_X=8", "-DLBM_BRICK_Y=4", "-DLBM_BRICK_Z=2")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + INCLUDE]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False, brick842: bool = False) -> str:
    """Builds the library (debug: the LBM_DEBUG variant; brick842: the 8 x 4 x 2 brick variant;
    each in its own folder) unless it is newer than every source; returns its path."""
    out_dir, lib = (DEBUG_OUT_DIR, DEBUG_LIB) if debug else (B842_OUT_DIR, B842_LIB) if brick842 else (OUT_DIR, LIB)
    if debug:
        extra_flags = ("-DLBM_DEBUG", *extra_flags)
    if brick842:
        extra_flags = (*B842_FLAGS, *extra_flags)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    objs = []
    procs = []
    for src in _sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((subprocess.Popen(cmd), src))
        objs.append(obj)
    failed = [src for p, src in procs if p.wait() != 0]
    if failed:
        raise RuntimeError("nvcc failed on: " + ", ".join(failed))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv,
                brick842="--brick842" in sys.argv,
                extra_flags=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []))
