"""Build libgmcp.so (the CUDA library behind include/gmcp.h) in-tree for
sm_103a with nvcc.  Run ``python -m paper_2605_24339_b300.build [-v] [-f]``."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgmcp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
# translation units whose FP64 predicates must round like a plain IEEE
# evaluation (no fused multiply-add): candidate boxes, CCD, and the sample
# geometry whose membership tests (point inside a slave triangle, edge
# clipping) are not weight-continuous and so must decide exactly as the
# CPU oracle does on degenerate (coincident) meshes
NO_FMA = {"broadphase.cu", "contact.cu", "faceclip.cu"}
SOURCES = ["api.cu", "scan.cu", "broadphase.cu", "contact.cu", "newton.cu", "warmstart.cu", "dualmap.cu",
           "faceclip.cu", "snapshot.cu", "peaks.cu"]


def nvcc() -> str:
    env = os.environ.get("NVCC")
    if env:
        return env
    return "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "gmcp.h"))
    objs, cmds = [], []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc(), *ARCH, *COMMON, "-c", path, "-o", obj]
            if src in NO_FMA:
                cmd.insert(1, "-fmad=false")
            if verbose:
                cmd += ["-Xptxas", "-v"]
                print(" ".join(cmd), flush=True)
            cmds.append(cmd)
    # translation units compile independently: run them side by side
    with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as pool:
        for f in [pool.submit(subprocess.check_call, cmd) for cmd in cmds]:
            f.result()
    if force or _stale(LIB, objs):
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lcudart",
                               "-Xlinker", "--no-undefined"])
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
