"""Build the in-tree CUDA library ``libhestonmc.so`` for sm_103a with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
SOURCES = [os.path.join(_HERE, "csrc", "heston_mc.cu")]
HEADERS = [os.path.join(_ROOT, "include", "heston_mc.h"), os.path.join(_HERE, "csrc", "heston_device.cuh")]
TARGET = os.path.join(_HERE, "libhestonmc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(p) for p in SOURCES + HEADERS)
    if not force and os.path.exists(TARGET) and os.path.getmtime(TARGET) >= newest:
        return TARGET
    tmp = TARGET + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(_ROOT, "include"), *SOURCES, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stderr[-4000:])
    os.replace(tmp, TARGET)
    return TARGET


if __name__ == "__main__":
    print(build(force=True, verbose=True))
