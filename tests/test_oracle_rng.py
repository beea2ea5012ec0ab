"""Pins of the oracle's Philox4x32-10 stream (CPU only).

The comparator is NVIDIA cuRAND's host-side PHILOX4_32_10 generator, run as a
library on the CPU: its output block b is Philox4x32-10 of counter
(b // 65536, 0, b % 65536, 0) under key (seed low, seed high).  Agreement over
tens of thousands of blocks and several keys pins the round function, the
multipliers, the Weyl key schedule and the word order.
"""
import ctypes as C
import os

import numpy as np
import pytest
from scipy import stats

CURAND = "/usr/local/cuda/lib64/libcurand.so.10"


def _curand_host_words(seed, n_words):
    if not os.path.exists(CURAND):
        pytest.skip("cuRAND not present")
    cr = C.CDLL(CURAND)
    g = C.c_void_p()
    assert cr.curandCreateGeneratorHost(C.byref(g), 161) == 0  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert cr.curandSetPseudoRandomGeneratorSeed(g, C.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert cr.curandGenerate(g, out.ctypes.data_as(C.c_void_p), C.c_size_t(n_words)) == 0
    finally:
        cr.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


@pytest.mark.parametrize("seed", [1, 0xDEADBEEF, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(orc, seed):
    blocks = _curand_host_words(seed, 4 * 65536 + 4 * 512)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    idx = list(range(0, 64)) + list(range(65500, 65536 + 512, 7))
    for b in idx:
        ctr = [b // 65536, 0, b % 65536, 0]
        assert orc.philox(ctr, key) == list(blocks[b]), (seed, b)


def test_philox_million_words_match_curand(orc):
    """2^20 consecutive words of cuRAND's host generator (blocks 0 .. 2^18 - 1),
    all of them: block b = r + 65536 j has counter (j, 0, r, 0), which is word
    4j.. of the oracle's stream of history r * 2^32, instance 0."""
    seed = 0x0123456789ABCDEF
    blocks = _curand_host_words(seed, 4 * 262144)
    for r in range(65536):
        w = orc.stream_words(seed, r << 32, 0, 16).reshape(4, 4)
        if not np.array_equal(w, blocks[r::65536]):
            raise AssertionError("block %d + 65536 j differs" % r)


def test_uniform_exact_and_open_interval(orc):
    for x in (0, 1, 511, 512, 0x7FFFFFFF, 0xFFFFFFFF):
        u = orc.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u      # 24 significant bits: identical in FP32
    assert orc.u01(0) == 2.0 ** -24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_stream_layout(orc):
    """Stream of (seed, history, instance): block n = Philox(n, hid lo, hid hi, inst)."""
    seed, hid, inst = 0x1122334455667788, 0x0000000A_00000003, 7
    w = orc.stream_words(seed, hid, inst, 12)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for n in range(3):
        assert list(w[4 * n:4 * n + 4]) == orc.philox([n, hid & 0xFFFFFFFF, hid >> 32, inst], key)


def test_uniformity_and_independence(orc):
    w = np.concatenate([orc.stream_words(1, h, 0, 64) for h in range(4000)])
    u = (2.0 * (w >> 9) + 1.0) * 2.0 ** -24
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-3
    # adjacent-pair correlation and history-to-history correlation
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01
    a = np.array([orc.stream_words(1, h, 0, 1)[0] for h in range(2000)], dtype=np.float64)
    b = np.array([orc.stream_words(1, h, 1, 1)[0] for h in range(2000)], dtype=np.float64)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.08
