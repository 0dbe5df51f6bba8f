"""Pins for the oracle's Philox4x32-10 (the counter-based RNG both sides use).

The oracle's generator is checked against cuRAND's host-side Philox4x32-10
generator (a library routine, called through its C API): cuRAND's host stream
for seed s and offset o emits, as its g-th 4-word block, Philox4x32-10 with key
(s_lo, s_hi) and counter ((g >> 16) mod 2^32, g >> 48, g & 0xffff, 0).  That
exercises both key words and counter words 0-2; word 3 is covered by the GPU
test against cuRAND's device function.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10"]
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_blocks(L, seed, offset, nblocks):
    gen = ctypes.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert L.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 12345, 0xDEADBEEFCAFEF00D])
@pytest.mark.parametrize("offset_blocks", [0, 100, 65530, 2**32 + 7, 2**48 + 70000])
def test_philox_matches_curand_host(seed, offset_blocks):
    L = _curand()
    if L is None:
        pytest.skip("libcurand not found")
    blocks = _curand_host_blocks(L, seed, 4 * offset_blocks, 8)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(8):
        g = offset_blocks + i
        ctr = [(g >> 16) & 0xFFFFFFFF, (g >> 48) & 0xFFFFFFFF, g & 0xFFFF, 0]
        assert list(oracle.philox(key, ctr)) == list(blocks[i]), (seed, g)


def test_philox_counter_words_all_matter():
    """each counter word and key word changes the output (no word is ignored)"""
    base = oracle.philox([1, 2], [3, 4, 5, 6])
    for w in range(4):
        c = [3, 4, 5, 6]
        c[w] ^= 1
        assert list(oracle.philox([1, 2], c)) != list(base)
    for w in range(2):
        k = [1, 2]
        k[w] ^= 1
        assert list(oracle.philox(k, [3, 4, 5, 6])) != list(base)


def test_philox_uniformity():
    """top-byte histogram of 4 x 20000 words over the (id, step, stream) layout is flat"""
    words = np.concatenate([oracle.philox([7, 0], [i, 0, 3, 2]) for i in range(20000)])
    hist = np.bincount(words >> 24, minlength=256)
    exp = words.size / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    # 255 degrees of freedom: mean 255, sd 22.6; 6 sd bound
    assert chi2 < 255 + 6 * 22.6
    bits = np.unpackbits(words.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.003
