"""The issue-rate micro-benchmarks behind the roofline denominators
(libpipepeaks.so, paper_2309_10477_gb300/peaks.py).

CPU: the library loads, names its kinds, and rejects bad arguments before
any CUDA call.  GPU: every kind runs; the FP32 FMA rate is one
thread-instruction per lane per clock (the issue rate) and the highest of the
single kinds; the f32x2 FMA rate is half of it; the FMA-pipe mix of the path
kernel (15 wide multiplies per 44 f32x2 FMAs) is no faster than either of its
parts alone allows; and the same FP32 work as scalar FFMAs costs the sum of
its parts (scalar FFMAs do not run beside the wide multiplies), which is why
the path kernel packs its FP32 work into f32x2 instructions."""
import ctypes
import os

import pytest

from paper_2309_10477_gb300 import peaks

KINDS = ["ffma", "ffma2", "imad_wide", "lop3", "mufu_ex2", "mufu_lg2", "mufu_sin", "mufu_cos",
         "mufu_rsqrt", "mufu_sqrt", "dfma", "imad_lo", "imad_hi", "heavy_mix", "scalar_mix"]


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(peaks._LIB):
        from paper_2309_10477_gb300 import build
        build.build()
    return peaks.load()


def test_library_names_its_kinds(lib):
    assert peaks.kinds() == KINDS
    assert lib.pipe_peak_name(-1) == b"" and lib.pipe_peak_name(len(KINDS)) == b""


def test_bad_arguments_are_rejected_before_any_launch(lib):
    n = ctypes.c_double()
    sink = ctypes.c_void_p(16)        # never dereferenced: the checks come first
    for kind, blocks, threads in ((-1, 1, 32), (len(KINDS), 1, 32), (0, 0, 32), (0, 1, 0), (0, 1, 2048)):
        assert lib.pipe_peak_launch(kind, blocks, threads, 1, None, sink, ctypes.byref(n)) == -1
    assert lib.pipe_peak_launch(0, 1, 32, 1, None, None, ctypes.byref(n)) == -1


@pytest.mark.gpu
def test_rates_are_consistent(lib):
    import torch
    r = peaks.measure(0.05)
    assert set(r) == set(KINDS)
    rate = {k: v["thread_insts_per_s"] for k, v in r.items()}
    assert all(v > 0 for v in rate.values())
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    # one FP32 FMA per lane per clock, 128 lanes per SM, at 1.0-2.2 GHz
    per_sm_clk_max = rate["ffma"] / (n_sm * 1.0e9)
    assert 0.85 * 128 * 1.0 <= per_sm_clk_max <= 1.02 * 128 * 2.2
    single = {k: v for k, v in rate.items() if not k.endswith("_mix")}
    assert max(single, key=single.get) == "ffma"
    assert 0.45 <= rate["ffma2"] / rate["ffma"] <= 0.55
    # the mix: a unit of 15 wide multiplies and 44 f32x2 FMAs takes at least as
    # long as either part alone at its own rate
    unit = rate["heavy_mix"] / 59.0
    assert unit <= 1.02 / max(15.0 / rate["imad_wide"], 44.0 / rate["ffma2"])
    # the scalar mix: 15 wide multiplies and 88 FFMAs take at least 0.9 of the
    # sum of their times alone, and no less time than the packed mix
    t_scalar = 103.0 / rate["scalar_mix"]
    assert t_scalar >= 0.9 * (15.0 / rate["imad_wide"] + 88.0 / rate["ffma"])
    assert t_scalar >= 0.95 * (59.0 / rate["heavy_mix"])
