"""Measured issue rates of the pipes the path kernels use (libpipepeaks.so).

Each instruction kind (FP32 FMA, f32x2 FMA, the wide 32x32->64 multiply and
the three-way xor of Philox, special-function-unit approximations, FP64 FMA)
runs in independent chains on every SM at full occupancy; a launch is timed
with CUDA events on the stream it runs on, and the rate is the executed
thread-instructions of that kind per second.  These rates are the roofline
denominators of the path kernels: the issue rate of the machine, the rate of
the pipe a kernel is bound by, and the FP64 rate that bounds the FP64 path.

    python -m paper_2309_10477_gb300.peaks [--seconds S]

prints the rates as JSON (the committed record under profiles/ comes from it).
"""
from __future__ import annotations

import ctypes
import json
import os
import statistics
import time

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libpipepeaks.so")
_lib = None

THREADS = 256
BLOCKS_PER_SM = 8          # 2048 threads per SM: full occupancy at <= 32 registers


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise RuntimeError(f"{_LIB} is not built: run paper_2309_10477_gb300.build.build()")
        lib = ctypes.CDLL(_LIB)
        lib.pipe_peak_kinds.restype = ctypes.c_int
        lib.pipe_peak_name.restype = ctypes.c_char_p
        lib.pipe_peak_name.argtypes = [ctypes.c_int]
        lib.pipe_peak_launch.restype = ctypes.c_int
        lib.pipe_peak_launch.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        _lib = lib
    return _lib


def kinds():
    lib = load()
    return [lib.pipe_peak_name(k).decode() for k in range(lib.pipe_peak_kinds())]


def measure(seconds_per_kind: float = 0.3, device: int = 0, only=None):
    """{kind: {"thread_insts_per_s", "ms_per_launch", "launches"}}: the median
    rate over launches of about 20 ms each, timed with CUDA events."""
    import torch
    lib = load()
    dev = torch.device("cuda", device)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = n_sm * BLOCKS_PER_SM
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    insts = ctypes.c_double()
    out = {}
    for k, name in enumerate(kinds()):
        if only and name not in only:
            continue

        def launch(iters):
            rc = lib.pipe_peak_launch(k, blocks, THREADS, iters, ctypes.c_void_p(stream.cuda_stream),
                                      ctypes.c_void_p(sink.data_ptr()), ctypes.byref(insts))
            if rc != 0:
                raise RuntimeError(f"pipe_peak_launch({name}) failed: {rc}")
            return insts.value

        def timed(iters):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n = launch(iters)
            e1.record(stream)
            e1.synchronize()
            return n, e0.elapsed_time(e1)

        iters = 64
        timed(iters)                                     # warm-up (module load)
        _, ms = timed(iters)
        iters = max(16, int(iters * 20.0 / max(ms, 1e-3)))   # about 20 ms per launch
        rates, times = [], []
        t_end = time.perf_counter() + seconds_per_kind
        while len(rates) < 3 or time.perf_counter() < t_end:
            n, ms = timed(iters)
            rates.append(n / (ms * 1e-3))
            times.append(ms)
        out[name] = {"thread_insts_per_s": statistics.median(rates),
                     "ms_per_launch": statistics.median(times), "launches": len(rates)}
    return out


def per_sm_clock(rates: dict, n_sm: int, sm_mhz: float):
    """The same rates as thread-instructions per SM per clock at sm_mhz."""
    return {k: v["thread_insts_per_s"] / (n_sm * sm_mhz * 1e6) for k, v in rates.items()}


if __name__ == "__main__":
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=2.0, help="timed seconds per kind")
    a = ap.parse_args()
    r = measure(a.seconds)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    print(json.dumps({"n_sm": n_sm, "rates": r}, indent=1))
