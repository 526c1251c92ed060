"""Pins for the oracle's Philox4x32-10 and Box-Muller normals.

The oracle's generator is checked against an independent implementation:
cuRAND's host-side PHILOX4_32_10 generator, called as a black box (it runs on
the CPU, no GPU needed).  Its output stream places block b at counter
(b // 65536, 0, b % 65536, 0) with key = (seed_lo, seed_hi); large generator
offsets reach counter word 1.  Normal draws are checked by their moments.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest

import oracle as O

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def curand_host_words(lib, seed, offset, n):
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def _ctr_for_block(b):
    b = np.asarray(b, dtype=np.uint64)
    hi = b // np.uint64(65536)
    return np.stack([hi & np.uint64(0xFFFFFFFF), hi >> np.uint64(32),
                     b % np.uint64(65536), np.zeros_like(b)], axis=-1)


@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEFCAFEBABE, 2**64 - 1])
def test_philox_matches_curand_stream(seed):
    lib = _curand()
    nblk = 70000                       # crosses the 65536-block boundary (word 0 = 1)
    w = curand_host_words(lib, seed, 0, 4 * nblk).reshape(nblk, 4)
    ctr = _ctr_for_block(np.arange(nblk, dtype=np.uint64))
    out = O.philox4x32_10(ctr, O.philox.seed_key(seed))
    assert np.array_equal(out, w)


@pytest.mark.parametrize("block", [65536 * 12345 + 17, 65536 * ((1 << 32) + 5) + 7,
                                   65536 * ((1 << 40) + 99) + 65535])
def test_philox_matches_curand_high_counter_words(block):
    lib = _curand()
    seed = 0x0123456789ABCDEF
    w = curand_host_words(lib, seed, 4 * block, 8).reshape(2, 4)
    ctr = _ctr_for_block(np.array([block, block + 1], dtype=np.uint64))
    assert np.array_equal(O.philox4x32_10(ctr, O.philox.seed_key(seed)), w)


def test_uniform_map_open_interval():
    u = O.uniforms_from_words(np.array([0, 2**32 - 1], dtype=np.uint64))
    assert u[0] == 0.5 * 2.0 ** -32
    assert 0.0 < u[0] < u[1] < 1.0
    assert u[1] == 1.0 - 0.5 * 2.0 ** -32


def test_normal_moments():
    n = 200_000
    eps = O.control_noise(seed=7, k=3, samples=np.arange(n), it=11, sigma=(1.0, 1.0))
    for c in range(2):
        z = eps[:, c]
        se = 1.0 / np.sqrt(n)
        assert abs(z.mean()) < 5 * se
        assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0) * se
        kurt = np.mean(z ** 4) / z.var() ** 2
        assert abs(kurt - 3.0) < 5 * np.sqrt(24.0) * se
    # the two components are uncorrelated
    assert abs(np.corrcoef(eps[:, 0], eps[:, 1])[0, 1]) < 5.0 / np.sqrt(n)


def test_normal_distribution_ks():
    scipy_stats = pytest.importorskip("scipy.stats")
    eps = O.control_noise(seed=3, k=0, samples=np.arange(50_000), it=0, sigma=(0.5, 0.8))
    assert scipy_stats.kstest(eps[:, 0] / 0.5, "norm").pvalue > 1e-3
    assert scipy_stats.kstest(eps[:, 1] / 0.8, "norm").pvalue > 1e-3


def test_counter_words_are_independent_streams():
    a = O.control_noise(seed=1, k=0, samples=np.arange(64), it=0, sigma=(1, 1))
    b = O.control_noise(seed=1, k=1, samples=np.arange(64), it=0, sigma=(1, 1))
    c = O.control_noise(seed=1, k=0, samples=np.arange(64), it=1 << 32, sigma=(1, 1))
    d = O.control_noise(seed=2, k=0, samples=np.arange(64), it=0, sigma=(1, 1))
    for x in (b, c, d):
        assert not np.any(x == a)
