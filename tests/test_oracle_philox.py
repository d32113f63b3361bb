"""Pins of the oracle's counter-based noise (Sec. II-B sampling step).

The oracle's Philox4x32-10 is written from the SC'11 definition.  It is
pinned against NVIDIA's cuRAND host generator (run as a black box on the CPU:
its Philox4_32_10 stream with seed s yields block i = Philox(key = s,
counter = (0, 0, i, 0))), and the normals against their distribution.
"""
import ctypes
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for path in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(path)
        except OSError:
            continue
    return None


def _curand_host_words(lib, seed, n_words):
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 7, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_stream(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    n_blocks = 2048
    words = _curand_host_words(lib, seed, 4 * n_blocks).reshape(n_blocks, 4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n_blocks):
        got = oracle.philox4x32_10([0, 0, i, 0], key)
        assert np.array_equal(got, words[i]), (hex(seed), i)


@pytest.mark.parametrize("seed", [7, 0x0123456789ABCDEF])
def test_normals_match_curand_host_normals(seed):
    """cuRAND's host normal generator on the Philox4_32_10 stream turns each
    block i (our counter (0, 0, i, 0): sample i at step 0, counter 0) into
    two Box-Muller pairs, emitting (r sin, r cos) where the solve's mapping
    emits (r cos, r sin); its uniform map differs from ours by at most
    2^-33, so the normals agree to ~1e-6."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not found")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    n_blocks = 1024
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.float32)
        assert lib.curandGenerateNormal(gen, out.ctypes.data_as(ctypes.c_void_p),
                                        ctypes.c_size_t(out.size), ctypes.c_float(0.0),
                                        ctypes.c_float(1.0)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    cur = out.reshape(n_blocks, 4)[:, [1, 0, 3, 2]].astype(np.float64)
    ours = np.array([oracle.normals(seed, 0, s, 0, 4) for s in range(n_blocks)])
    assert np.max(np.abs(cur - ours)) < 2e-5


def test_philox_is_a_bijection_sample():
    # distinct counters give distinct outputs (a permutation for fixed key)
    key = [0xDEADBEEF, 0x12345678]
    seen = set()
    for a in range(16):
        for b in range(16):
            seen.add(tuple(oracle.philox4x32_10([a, b, 3, 9], key)))
    assert len(seen) == 256


def test_normals_distribution():
    # 40k normals from the solve's noise mapping: N(0, 1) by KS, moments,
    # and no correlation between the two halves of a Box-Muller pair.
    d = 8
    vals = np.array([oracle.normals(11, 5, s, tau, d) for s in range(500) for tau in range(10)])
    flat = vals.reshape(-1)
    assert abs(flat.mean()) < 5.0 / np.sqrt(flat.size)
    assert abs(flat.var() - 1.0) < 5.0 * np.sqrt(2.0 / flat.size)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    r = np.corrcoef(vals[:, 0], vals[:, 1])[0, 1]
    assert abs(r) < 5.0 / np.sqrt(vals.shape[0])  # 5 sigma
    # lanes of one block and blocks of one step are distinct streams
    assert not np.allclose(vals[:, 0], vals[:, 4])


def test_normals_positional():
    # normal q depends only on (seed, counter, s, tau, q): drawing more
    # components does not change the first ones.
    a = oracle.normals(3, 1, 17, 4, 5)
    b = oracle.normals(3, 1, 17, 4, 68)
    assert np.array_equal(a, b[:5])
    # the counter's low 32 bits select the stream
    c = oracle.normals(3, 1 + (1 << 32), 17, 4, 5)
    assert np.array_equal(a, c)
    assert not np.array_equal(a, oracle.normals(3, 2, 17, 4, 5))


def test_normals_extreme_words_finite():
    # the uniform map keeps u in (0, 1): log never sees 0, so every normal is
    # finite and bounded by sqrt(-2 ln 2^-24) ~ 5.77.
    vals = np.array([oracle.normals(s, 0, 0, 0, 4) for s in range(2000)])
    assert np.all(np.isfinite(vals))
    assert np.abs(vals).max() < math.sqrt(-2.0 * math.log(2.0**-24)) + 1e-9
