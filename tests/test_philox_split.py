"""The path kernel's split Philox4x32-10 (csrc/philox.cuh: the warp-uniform
(step pair, high path word) part of its first three rounds computed once per warp, the
rest per path) gives the same words as the plain ten rounds, and both equal
the oracle's Philox4x32-10 (itself pinned to cuRAND's host generator).
Compiled here as a host program; no GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_10477_gb300", "csrc")


@pytest.fixture(scope="module")
def check_exe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("philox") / "philox_split_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                    os.path.join(ROOT, "tests", "native", "philox_split_check.cu")],
                   check=True, capture_output=True)
    return exe


def _cases():
    rng = np.random.default_rng(20230918)
    n = 4000
    j = rng.integers(0, 2**32, n, dtype=np.uint64)
    j[: n // 2] %= 4096                          # step pairs as the kernels use them
    p = rng.integers(0, 2**32, n, dtype=np.uint64)
    h = rng.integers(0, 2**32, n, dtype=np.uint64)
    h[: n // 4] = 0                              # paths below 2^32
    h[n // 4: n // 2] = 1
    k = rng.integers(0, 2**32, (n, 2), dtype=np.uint64)
    edge = np.array([[0, 0, 0, 0, 0], [2**32 - 1] * 5, [125, 2**32 - 1, 0, 42, 0]], dtype=np.uint64)
    return np.vstack([np.column_stack([j, p, h, k]), edge])


def test_split_equals_plain_rounds_and_oracle(check_exe):
    cases = _cases()
    inp = "\n".join(" ".join(str(int(x)) for x in row) for row in cases) + "\n"
    out = subprocess.run([check_exe], input=inp, capture_output=True, text=True, check=True).stdout
    words = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()])
    assert words.shape == (len(cases), 8)
    assert (words[:, :4] == words[:, 4:]).all()
    for row, w in zip(cases[::40], words[::40]):
        j, p, h, k0, k1 = (int(x) for x in row)
        assert oracle.philox4x32_10([j, p, h, 0], [k0, k1]) == [int(x) for x in w[:4]]
