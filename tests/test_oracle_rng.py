"""Pins for the oracle's random-number contract (Philox4x32-10 + Box-Muller).

The Philox block function is pinned to an independent implementation:
cuRAND's host-side PHILOX4_32_10 generator, run (not read) on the CPU.  Its
output stream is block b = 65536*j + t with counter (j, 0, t, 0) and key
(seed_lo, seed_hi), which fixes the round function, the key schedule and
the placement of key and counter words.  The normals are pinned to the
standard normal law (moments, KS against scipy's CDF).
"""
import ctypes
import os

import numpy as np
import pytest
from scipy import stats

import oracle

CURAND = "/usr/local/cuda/lib64/libcurand.so"


def _curand_host_stream(seed, n_words):
    if not os.path.exists(CURAND):
        pytest.skip("libcurand not installed")
    lib = ctypes.CDLL(CURAND)
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0   # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 42, 0x0123456789ABCDEF, 2**64 - 1])
def test_philox_block_matches_curand_host_generator(seed):
    blocks = _curand_host_stream(seed, 4 * 65536 * 3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for b in list(range(0, 300)) + [65535, 65536, 65537, 70000, 131072 + 12345, 196607]:
        j, t = divmod(b, 65536)
        assert oracle.philox4x32_10([j, 0, t, 0], key) == [int(x) for x in blocks[b]], b


def test_uniform_mapping_is_24_bit_and_in_range():
    seed = 42
    for path in (0, 1, 2**32 + 5):
        for step in range(0, 9):
            u1, u2 = oracle.uniform_pair(seed, path, step)
            words = oracle.philox4x32_10([step // 2, path & 0xFFFFFFFF, path >> 32, 0],
                                         [seed & 0xFFFFFFFF, seed >> 32])
            a, b = (words[2], words[3]) if step & 1 else (words[0], words[1])
            assert u1 == ((a >> 8) + 1) / 2**24
            assert u2 == (b >> 8) / 2**24
            assert 0.0 < u1 <= 1.0 and 0.0 <= u2 < 1.0


def test_stream_tag_changes_draws():
    a = oracle.uniform_pair(7, 3, 4, 0)
    b = oracle.uniform_pair(7, 3, 4, 2)
    assert a != b


def test_box_muller_normals_are_standard_normal():
    n_paths, n_steps = 4096, 256
    za = np.empty((n_paths, n_steps))
    zb = np.empty((n_paths, n_steps))
    for i in range(n_paths):
        za[i], zb[i] = oracle.path_normals(42, i, n_steps)
    for z in (za.ravel(), zb.ravel()):
        n = z.size
        assert abs(z.mean()) < 5 / np.sqrt(n)
        assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
        assert abs(stats.skew(z)) < 5 * np.sqrt(6.0 / n)
        assert abs(stats.kurtosis(z)) < 5 * np.sqrt(24.0 / n)
        assert stats.kstest(z, "norm").pvalue > 1e-4
    # the two normals of a pair, and consecutive steps, are uncorrelated
    assert abs(np.corrcoef(za.ravel(), zb.ravel())[0, 1]) < 5 / np.sqrt(za.size)
    assert abs(np.corrcoef(za[:, :-1].ravel(), za[:, 1:].ravel())[0, 1]) < 5 / np.sqrt(za.size)
    # the largest |Z| a 24-bit u1 allows is sqrt(2 * 24 ln 2)
    assert np.abs(za).max() <= np.sqrt(-2 * np.log(2.0**-24)) + 1e-12
