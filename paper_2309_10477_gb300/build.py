"""Build the in-tree CUDA libraries for sm_103a with nvcc: ``libhestonmc.so``
(the pricing path behind include/heston_mc.h) and ``libpipepeaks.so`` (the
issue-rate micro-benchmarks that give the roofline denominators).  The two
compile in parallel."""
from __future__ import annotations

import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
SOURCES = [os.path.join(_HERE, "csrc", "heston_mc.cu")]
HEADERS = [os.path.join(_ROOT, "include", "heston_mc.h"), os.path.join(_HERE, "csrc", "heston_device.cuh"),
           os.path.join(_HERE, "csrc", "philox.cuh"),
           os.path.join(_HERE, "csrc", "bm64_tables.h")]
TARGET = os.path.join(_HERE, "libhestonmc.so")
PEAKS_SOURCES = [os.path.join(_HERE, "csrc", "pipe_peaks.cu")]
PEAKS_TARGET = os.path.join(_HERE, "libpipepeaks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    return not os.path.exists(target) or os.path.getmtime(target) < max(os.path.getmtime(p) for p in deps)


def _cmd(sources, tmp, verbose):
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-I", os.path.join(_ROOT, "include"), *sources, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def build(force: bool = False, verbose: bool = False) -> str:
    jobs = []
    for sources, deps, target in ((SOURCES, SOURCES + HEADERS, TARGET),
                                  (PEAKS_SOURCES, PEAKS_SOURCES, PEAKS_TARGET)):
        if force or _stale(target, deps):
            tmp = target + f".tmp{os.getpid()}"
            p = subprocess.Popen(_cmd(sources, tmp, verbose), stdout=subprocess.PIPE,
                                 stderr=subprocess.PIPE, text=True)
            jobs.append((p, tmp, target))
    for p, tmp, target in jobs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(target)}:\n" + err[-4000:])
        if verbose:
            print(err)
        os.replace(tmp, target)
    return TARGET


if __name__ == "__main__":
    print(build(force=True, verbose=True))
