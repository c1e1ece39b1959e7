"""Pins for the oracle's Philox4x32-10 (published definition, SC'11).

The independent reference is NVIDIA's cuRAND host-side PHILOX4_32_10
generator, run through its public C API with ctypes (run, never read).  Its
output stream was found to lay out 4-word blocks so that global block b is
the Philox block with key (seed_lo, seed_hi) and counter
(b div 65536, 0, b mod 65536, 0); the test checks the oracle against that
layout, which exercises both key words and counter words 0 and 2.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

from oracle import philox

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = []
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    for sub in ("lib64", "lib", "targets/sbsa-linux/lib", "targets/x86_64-linux/lib"):
        cands += [os.path.join(cuda, sub, "libcurand.so"), os.path.join(cuda, sub, "libcurand.so.10")]
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_words(lib, seed, offset_words, n_words):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    key = philox.split_seed(seed)
    for first_block, n_blocks in [(0, 2048), (65536 - 8, 16), (3 * 65536 + 17, 64)]:
        words = _curand_host_words(lib, seed, 4 * first_block, 4 * n_blocks).reshape(-1, 4)
        b = np.arange(first_block, first_block + n_blocks, dtype=np.uint64)
        ctr = np.zeros((n_blocks, 4), dtype=np.uint64)
        ctr[:, 0] = b >> np.uint64(16)
        ctr[:, 2] = b & np.uint64(0xFFFF)
        mine = philox.philox4x32_10(ctr, key)
        np.testing.assert_array_equal(mine, words)


def test_philox_is_a_bijection_on_a_sample():
    # distinct counters under one key give distinct blocks (Philox is a bijection)
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(20000, 4), dtype=np.uint64)
    ctr = np.unique(ctr, axis=0)
    out = philox.philox4x32_10(ctr, philox.split_seed(7))
    assert np.unique(out, axis=0).shape[0] == ctr.shape[0]


def test_philox_word_uniformity():
    ctr = np.zeros((1 << 16, 4), dtype=np.uint64)
    ctr[:, 1] = np.arange(1 << 16)
    ctr[:, 3] = 5
    w = philox.philox4x32_10(ctr, philox.split_seed(42)).astype(np.uint64)
    # every bit of every word is set with probability 1/2
    bits = np.stack([(w >> np.uint64(i)) & np.uint64(1) for i in range(32)], axis=-1).astype(np.float64)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 5 * 0.5 / np.sqrt(w.shape[0]))


def test_split_seed():
    np.testing.assert_array_equal(philox.split_seed(0x0123456789ABCDEF), [0x89ABCDEF, 0x01234567])
