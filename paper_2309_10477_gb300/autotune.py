"""Launch-shape autotuner for the persistent batched kernel and the
single-contract path kernel.

Results do not depend on the launch shape (tile rows are fixed by the path
index), so the tuner may try any shape: it times each candidate (block
threads, CTAs per SM) with CUDA events on the caller's stream, keeps the
fastest, and caches the choice per problem key for the process.
"""
from __future__ import annotations

import statistics

import torch

from . import native

_cache: dict = {}


def candidates(n_sm: int, blocks=(64, 128), ctas_per_sm=(2, 3, 4, 5, 6, 7, 8, 10, 12, 14)):
    """(block_threads, grid_ctas) pairs; grid 0 lets the library size the grid."""
    out = [(b, 0) for b in blocks]
    for b in blocks:
        for c in ctas_per_sm:
            if b * c <= 2048:
                out.append((b, n_sm * c))
    return out


def tune(key, launch, cands, reps: int = 3, stream=None):
    """launch(block_threads, grid_ctas) enqueues one run.  Returns the best
    (block, grid) and the timings (ms); cached under `key`."""
    if key in _cache:
        return _cache[key]
    stream = stream or torch.cuda.current_stream()
    timings = {}
    for b, g in cands:
        launch(b, g)                                       # warm-up, also checks the shape
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch(b, g)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        timings[(b, g)] = statistics.median(ts)
    best = min(timings, key=timings.get)
    _cache[key] = (best, timings)
    return best, timings


def tune_batch(plan, desc, workspace, out, base_options, stream=None, reps: int = 2):
    """Best (block_threads, grid_ctas) for a prepared batch."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    key = ("batch", int(plan.n_items), int(plan.total_tiles).bit_length(), int(plan.trunc))

    def launch(b, g):
        o = native.heston_options.from_buffer_copy(base_options)
        o.block_threads, o.grid_ctas = b, g
        native.heston_mc_launch_batch(plan, desc, o, workspace, out)

    return tune(key, launch, candidates(n_sm), reps=reps, stream=stream)
