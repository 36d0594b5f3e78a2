"""Build step of the solver's shared library (nvcc, sm_103a only).

``python -m paper_2408_12179_b300.build`` compiles ``csrc/hpr_api.cu`` (which includes
the device code in ``csrc/hpr_device.cuh``) into ``libhpr_b300.so`` beside this file:
one C-ABI shared object with no torch dependency, the CUDA runtime linked statically.
``build_checked`` compiles the same sources with HPR_BOUNDS_CHECK into
``libhpr_b300_checked.so``: every gather's index is checked against its vector's length
and out-of-range indices are counted (hpr_bounds_violations) instead of being loaded.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = [os.path.join(HERE, "csrc", "hpr_api.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", "hpr_device.cuh"), os.path.join(HERE, "csrc", "hpr_mlp.cuh"),
              os.path.join(HERE, "csrc", "hpr_small.cuh"), os.path.join(HERE, "csrc", "hpr_grid.cuh"),
              os.path.join(HERE, "csrc", "hpr_cluster.cuh"), os.path.join(HERE, "csrc", "hpr_tiles.cuh"),
              *(os.path.join(HERE, "csrc", f"hpr_api_{part}.cuh") for part in ("solve", "batch", "policy", "noalloc", "probe")),
              os.path.join(ROOT, "include", "hpr.h")]
LIB = os.path.join(HERE, "libhpr_b300.so")
LIB_CHECKED = os.path.join(HERE, "libhpr_b300_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_cmd(out=LIB, extra=()):
    return [NVCC, *ARCH, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
            "-shared", "-I", os.path.join(ROOT, "include"), "-o", out, *SRC, *extra]


def _build(out, force, extra):
    if not force and os.path.exists(out):
        newest = max(os.path.getmtime(p) for p in DEPS)
        if os.path.getmtime(out) >= newest:
            return out
    subprocess.run(nvcc_cmd(out=out, extra=extra), check=True)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    return _build(LIB, force, ["-Xptxas", "-v"] if verbose else [])


def build_checked(force: bool = False) -> str:
    """The bounds-checking build (a test build: slower, same results when no index is out
    of range)."""
    return _build(LIB_CHECKED, force, ["-DHPR_BOUNDS_CHECK"])


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
    if "--checked" in sys.argv:
        print(build_checked(force=True))
