"""Pins for the oracle's Philox4x32-10 generator and the draw mapping.

The generator is Philox4x32-10 of Salmon, Moraes, Dror & Shaw (SC'11).  It is
pinned against cuRAND's host-side Philox4_32_10 generator, an independent
implementation whose output block b is the Philox block with counter
(c mod 2^32, c div 2^32, b mod 65536, 0), c = b div 65536, and key = the
64-bit seed's halves: from the start of the sequence and from generator
offsets far enough that the counter's second word is nonzero.  The fourth
counter word (the purpose of a draw) is 0 in that layout; it is covered by
the GPU's parity with the oracle on the purpose streams 1 to 3, two
implementations written apart.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    return None


def _curand_host_words(lib, seed, count, offset=0):
    gen = ctypes.c_void_p()
    philox = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), philox) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        buf = (ctypes.c_uint * count)()
        assert lib.curandGenerate(gen, buf, ctypes.c_size_t(count)) == 0
        return np.array(buf, dtype=np.uint32)
    finally:
        lib.curandDestroyGenerator(gen)


def _host_counter(b):
    c = b // 65536
    return [c & 0xFFFFFFFF, c >> 32, b % 65536, 0]


@pytest.mark.parametrize("seed", [1, 12345, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    nblk = 65536 + 64
    words = _curand_host_words(lib, seed, 4 * nblk)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(7)
    blocks = list(range(16)) + list(rng.integers(0, nblk, 48)) + [65535, 65536, 65537, nblk - 1]
    for b in blocks:
        b = int(b)
        got = oracle.philox4x32_10(_host_counter(b), key)
        assert (got == words[4 * b:4 * b + 4]).all(), (seed, b)


@pytest.mark.parametrize("seed,offset", [(7, 2**51 + 4 * 12345), (0x0123456789ABCDEF, 2**50), (2**64 - 3, 2**62),
                                         (99, 2**50 + 4 * (65536 - 8))])
def test_philox_matches_curand_host_far_offsets(seed, offset):
    # offset in 32-bit words: block b = offset / 4 + t, so the counter's
    # first word wraps and its second word is nonzero
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    nblk = 32
    words = _curand_host_words(lib, seed, 4 * nblk, offset)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(nblk):
        b = offset // 4 + t
        got = oracle.philox4x32_10(_host_counter(b), key)
        assert (got == words[4 * t:4 * t + 4]).all(), (seed, offset, t)
        assert _host_counter(b)[1] > 0


def test_draw_mapping_contract():
    # draw i: high word j = i mod 4 of block (i>>2, rep, cell, purpose), low
    # word j of block (i>>2, rep, cell, purpose + 2^31); m = h 2^21 + (l >> 11) + 1
    seed, cell, rep, purpose = 0xDEADBEEF12345678, 17, 99, 2
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in [0, 1, 2, 3, 4, 1001, 2**34 - 1]:
        wh = oracle.philox4x32_10([i >> 2, rep, cell, purpose], key)
        wl = oracle.philox4x32_10([i >> 2, rep, cell, purpose + 2**31], key)
        j = i & 3
        assert oracle.draw_m(seed, cell, rep, purpose, i) == (int(wh[j]) << 21) + (int(wl[j]) >> 11) + 1


def test_draw_low_bits_uniform():
    # the 21 low bits of m - 1 come from the second stream: uniform too
    n = 100_000
    ms = np.array([oracle.draw_m(3, 1, r, 1, i) for r in range(10) for i in range(n // 10)], dtype=np.uint64)
    low = ((ms - np.uint64(1)) & np.uint64(0xFF)).astype(np.int64)
    counts = np.bincount(low, minlength=256)
    exp = n / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 6 * 22.6


def test_draw_range_and_uniformity():
    # m in [1, 2^53]; top 8 bits of (m-1) uniform (chi-square, 255 dof)
    n = 200_000
    ms = np.array([oracle.draw_m(1, 0, r, 0, i) for r in range(20) for i in range(n // 20)],
                  dtype=np.uint64)
    assert ms.min() >= 1 and ms.max() <= 2**53
    top = ((ms - np.uint64(1)) >> np.uint64(45)).astype(np.int64)
    counts = np.bincount(top, minlength=256)
    exp = n / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    # 255 dof: mean 255, sd ~22.6; 6 sd bound
    assert chi2 < 255 + 6 * 22.6
    # low bit of m is unbiased too
    assert abs((ms & np.uint64(1)).mean() - 0.5) < 6 * 0.5 / np.sqrt(n)
