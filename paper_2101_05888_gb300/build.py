"""Builds libsas.so (the CUDA library behind include/sas.h) in the package
directory with nvcc for sm_103a.  Translation units compile in parallel; the
link uses the static CUDA runtime, so the library has no dependency beyond the
driver."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsas.so")
OUT_CHECKED = os.path.join(HERE, "libsas_checked.so")   # -DSAS_CHECKED: index checks report in the status word
BUILD_DIR = os.path.join(os.path.dirname(HERE), "_build")
SOURCES = ["sas_api.cu", "tdbp_forward.cu", "tdbp_vjp.cu", "tdbp_adjoint.cu", "sharpness.cu", "sharpness_static.cu", "mlp.cu",
           "simulate.cu", "condition.cu", "micronav.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _inputs():
    # every header in csrc/ and include/: an edit to any of them rebuilds the library
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                     glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h")))
    return [os.path.join(CSRC, s) for s in SOURCES] + headers + [__file__]


def up_to_date(checked: bool = False) -> bool:
    out = OUT_CHECKED if checked else OUT
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _compile(src: str, checked: bool = False) -> str:
    obj_dir = os.path.join(BUILD_DIR, "checked") if checked else BUILD_DIR
    obj = os.path.join(obj_dir, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *(["-DSAS_CHECKED"] if checked else []), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libsas.so, or with checked=True libsas_checked.so (the same
    sources with -DSAS_CHECKED); returns the library's path."""
    out = OUT_CHECKED if checked else OUT
    if not force and up_to_date(checked):
        return out
    os.makedirs(os.path.join(BUILD_DIR, "checked") if checked else BUILD_DIR, exist_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda src: _compile(src, checked), SOURCES))
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, out)
    if verbose:
        print("built", out, file=sys.stderr)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
