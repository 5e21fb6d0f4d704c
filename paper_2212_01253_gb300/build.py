"""Builds libmslice.so (sm_103a) in-tree with nvcc.

The slice-loop kernels are specialised per (ny, nz) and compiled in one
translation unit per row length, in parallel; the host/C-ABI unit is compiled
alongside, and the objects are linked into one shared library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
HEADER = os.path.join(ROOT, "include", "mslice.h")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libmslice.so")
ROW_LENGTHS = (64, 128, 256, 512, 1024)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmslice")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(CSRC, "*.h")) + [HEADER, os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _sources())


def _units():
    inc = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]
    units = [(os.path.join(CSRC, "mslice.cu"), os.path.join(BUILD_DIR, "mslice.o"), inc),
             (os.path.join(CSRC, "mslice_recon.cu"), os.path.join(BUILD_DIR, "mslice_recon.o"), inc),
             (os.path.join(CSRC, "mslice_nn.cu"), os.path.join(BUILD_DIR, "mslice_nn.o"), inc),
             (os.path.join(CSRC, "mslice_rotate.cu"), os.path.join(BUILD_DIR, "mslice_rotate.o"), inc),
             (os.path.join(CSRC, "mslice_tc.cu"), os.path.join(BUILD_DIR, "mslice_tc.o"), inc),
             (os.path.join(CSRC, "mslice_generic.cu"), os.path.join(BUILD_DIR, "generic_paraxial.o"),
              inc + ["-DMS_AS=0"]),
             (os.path.join(CSRC, "mslice_generic.cu"), os.path.join(BUILD_DIR, "generic_angular.o"),
              inc + ["-DMS_AS=1"])]
    for ny in ROW_LENGTHS:
        for a in (0, 1):   # paraxial one-pass / angular-spectrum two-pass instances
            units.append((os.path.join(CSRC, "mslice_inst.cu"),
                          os.path.join(BUILD_DIR, "inst_%sny%d.o" % ("as_" if a else "", ny)),
                          inc + ["-DMS_NY=%d" % ny, "-DMS_AS=%d" % a]))
    return units


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile the CUDA library for sm_103a; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    extra = ["-Xptxas=-v"] if verbose else []

    def compile_one(u):
        src, obj, flags = u
        cmd = [cc, *CFLAGS, *extra, *flags, "-c", "-o", obj, src]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (os.path.basename(obj), r.stdout))
        return obj, r.stdout

    units = _units()
    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, units))
    if verbose:
        for obj, out in results:
            print("==", os.path.basename(obj))
            print(out)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results] + ["-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
