"""Build libsif.so in-tree with nvcc for sm_103a (GB300).

The kernels that take the method's branch decisions (geometry, mixing,
extension, interface, level set) are compiled without FMA contraction so
that they round like the CPU reference; the hot finite-volume kernel keeps
contraction.  Translation units compile in parallel, then link.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libsif.so")
ROOT = os.path.dirname(HERE)

SOURCES = {
    "kernels_geom.cu": ["--fmad=false"],
    "kernels_band.cu": ["--fmad=false"],
    "kernels_plan.cu": ["--fmad=false"],
    "kernels_fv.cu": ["--fmad=true"],
    "api.cu": [],
    "probe.cu": ["--fmad=true"],
    "noalloc.cu": ["--fmad=false"],
    "adjoint.cu": ["--fmad=true"],
    "kernels3d.cu": ["--fmad=false"],
    "fv3d.cu": ["--fmad=true"],
    "api3d.cu": [],
}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsif")
    return p


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES]
    files += [os.path.join(CSRC, "sif_internal.cuh"), os.path.join(CSRC, "sif3d_internal.cuh"),
              os.path.join(CSRC, "weno_frac.cuh"),
              os.path.join(ROOT, "include", "sif.h"), os.path.join(ROOT, "include", "sif3d.h"),
              os.path.abspath(__file__)]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-rdc=false",
              "-I", os.path.join(ROOT, "include")] + ARCH + list(extra)
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc, "-c", src, "-o", obj] + common + SOURCES[name]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, "-shared", "-o", tmp] + [o for o, _ in results] + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
