"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The reference point is an independent implementation: libcurand's host-side
PHILOX4_32_10 generator.  For the first 65536 blocks its output block j is
Philox4x32-10 of counter (0, 0, j, 0) under key (seed_lo, seed_hi), so every
round, both multipliers and both Weyl key increments are exercised.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if path and (os.path.exists(path) or not path.startswith("/")):
            try:
                return ctypes.CDLL(path)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_libcurand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("curand host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        nblk = 512
        out = np.zeros(4 * nblk, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for j in range(nblk):
        got = oracle.philox4x32_10([0, 0, j, 0], key)
        assert list(got) == list(out[4 * j:4 * j + 4]), f"block {j}"


def test_philox_uniformity_chi2():
    """Top 8 bits of 2^16 x 4 words over photon-id counters: chi^2 over 256 bins."""
    key = [7, 11]
    words = np.concatenate([oracle.philox4x32_10([i, 0, 0, 0], key) for i in range(1 << 14)])
    hist = np.bincount(words >> 24, minlength=256)
    exp = words.size / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    # 255 dof: mean 255, sd ~22.6; 6 sd bound
    assert chi2 < 255 + 6 * 22.6


def test_philox_counter_words_all_matter():
    key = [3, 5]
    base = oracle.philox4x32_10([1, 2, 3, 4], key)
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        assert list(oracle.philox4x32_10(c, key)) != list(base)
    assert list(oracle.philox4x32_10([1, 2, 3, 4], [3, 4])) != list(base)
    assert list(oracle.philox4x32_10([1, 2, 3, 4], [2, 5])) != list(base)
