"""Pins for the oracle's random numbers.

Philox4x32-10 is checked against an implementation that is not ours: cuRAND's
host-side PHILOX4_32_10 generator (it runs on the CPU, no GPU needed).  With
seed s, its output block b is philox(counter = (p mod 2^32, p >> 32,
b mod 65536, 0), key = (s mod 2^32, s >> 32)) with p = b // 65536 + offset
blocks, which exercises both key words and counter words 0, 1 and 2.
"""
import ctypes
import ctypes.util
import math
import os

import numpy as np
import pytest

import oracle

CURAND_PATHS = ["/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10"]


def _curand():
    for p in CURAND_PATHS:
        if os.path.exists(p):
            return ctypes.CDLL(p)
    p = ctypes.util.find_library("curand")
    if p:
        return ctypes.CDLL(p)
    return None


def _curand_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, np.uint32)
        assert lib.curandGenerate(gen, ctypes.c_void_p(out.ctypes.data), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    words = _curand_words(lib, seed, 0, 4 * 300)
    for b in range(300):
        ref = words[4 * b:4 * b + 4]
        mine = oracle.philox_block(0, 0, b, 0, k0, k1)
        assert np.array_equal(ref, mine), (seed, b)


def test_philox_counter_words_0_and_1_match_curand_host():
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    seed = 0x243F6A8885A308D3
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    for pos in (1, 7, 12345, (1 << 32) + 5, (3 << 32) + 0xFFFFFFFF):
        for sub in (0, 17, 65535):
            block = pos * 65536 + sub
            words = _curand_words(lib, seed, 4 * block, 4)
            p0, p1 = pos & 0xFFFFFFFF, pos >> 32
            assert np.array_equal(words, oracle.philox_block(p0, p1, sub, 0, k0, k1)), (pos, sub)


def test_uniform_open_interval_and_layout():
    # uniform j uses block j // 2, words 2(j%2), 2(j%2)+1: top 52 bits + 1/2
    seed, tag, c0, c1, c2 = 12345, 4, 7, 9, 11
    for j in range(8):
        w = oracle.philox_block(c0, c1, c2, (tag << 24) | (j // 2), seed & 0xFFFFFFFF, seed >> 32)
        hi, lo = int(w[2 * (j % 2)]), int(w[2 * (j % 2) + 1])
        m = (hi << 20) | (lo >> 12)
        assert oracle.uniform(seed, tag, c0, c1, c2, j) == (m + 0.5) * 2.0 ** -52
    us = np.array([oracle.uniform(3, 1, i, 0, 0, 0) for i in range(20000)])
    assert us.min() > 0.0 and us.max() < 1.0
    # chi-square over 20 bins, 19 dof: 99.99% quantile ~ 50
    h, _ = np.histogram(us, bins=20, range=(0, 1))
    chi2 = ((h - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 50.0


def test_iround_mean_and_variance():
    # Sec. 3.2 step i: Iround(x) = floor(x)+1 w.p. x - floor(x); mean x,
    # variance f(1-f)
    rng = np.random.default_rng(0)
    for x in (0.0, 0.3, 2.75, 17.5):
        u = rng.random(200000)
        vals = np.array([oracle.iround(x, float(v)) for v in u[:50000]])
        f = x - math.floor(x)
        se = math.sqrt(f * (1 - f) / len(vals)) + 1e-12
        assert abs(vals.mean() - x) <= 4 * se + 1e-12
        assert set(np.unique(vals)).issubset({math.floor(x), math.floor(x) + 1})
        assert abs(vals.var() - f * (1 - f)) < 0.01
