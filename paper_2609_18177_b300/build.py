"""Build the lbmh CUDA library (C ABI) for sm_103a, in-tree.

    python -m paper_2609_18177_b300.build [--force]

Produces paper_2609_18177_b300/_lbmh.so from csrc/*.cu with nvcc; the
library exports the functions declared in include/lbmh.h.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "_lbmh.so")
# the same library with every global-memory index of the step kernels guarded
# (LBMH_CHECK_BOUNDS): an index outside its array sets a status bit and is
# clamped; for the debug runs of the test suite, not for timing
LIB_CHECKED = os.path.join(HERE, "_lbmh_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(ROOT, "include", "lbmh.h"), os.path.abspath(__file__)]


def up_to_date(target, inputs):
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(p) <= t for p in inputs)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    if not force and up_to_date(lib, deps()):
        return lib
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
           "-I", os.path.join(ROOT, "include"), "-o", lib + ".tmp", *sources(), "-lcuda"]
    if checked:
        cmd.insert(1, "-DLBMH_CHECK_BOUNDS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
