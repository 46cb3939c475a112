"""Build the CUDA library libfsi.so in-tree for sm_103a (nvcc, no cmake)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libfsi.so")
SOURCES = ["fsi.cu", "fsi3.cu", "batch.cpp"]
HEADERS = ["fsi_kernels.cuh", "fsi_tc.cuh", "fsi_element.cuh", "fsi_internal.h", "fsi_mesh3d.h", "fsi_element3d.cuh", "fsi_mg3d.h",
           "fsi_vanka3.h", os.path.join("..", "..", "include", "fsi.h")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for f in SOURCES + HEADERS:
        if os.path.getmtime(os.path.join(CSRC, f)) > t:
            return True
    return False


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile libfsi.so if it is missing or older than its sources; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    # one nvcc per translation unit, in parallel, then one link
    flags = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-pthread"]
    if verbose:
        flags.append("-Xptxas=-v")
    objs, procs = [], []
    for f in SOURCES:
        obj = os.path.join(LIBDIR, os.path.splitext(f)[0] + ".o")
        objs.append(obj)
        procs.append((f, subprocess.Popen([nvcc()] + flags + ["-c", os.path.join(CSRC, f), "-o", obj],
                                          stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    logs, failed = [], []
    for f, pr in procs:
        out, _ = pr.communicate()
        logs.append(out)
        if pr.returncode != 0:
            failed.append(f + ":\n" + out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    res = subprocess.run([nvcc(), ARCH, "-shared", "-Xcompiler", "-pthread", "-o", LIB + ".tmp"] + objs,
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    if verbose:
        print("".join(logs) + res.stdout + res.stderr)
    for o in objs:
        os.remove(o)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build_library(force=True, verbose="-v" in sys.argv))
