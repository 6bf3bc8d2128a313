"""Pins of the oracle's Philox-4x32-10 and of its uniform draws.

Philox-4x32-10 is defined by Salmon et al. (SC'11). The independent reference
is a library routine: cuRAND's host generator CURAND_RNG_PSEUDO_PHILOX4_32_10.
With 64-bit seed s it uses key (s mod 2^32, s div 2^32) and interleaves 65536
subsequences: stream word 4 (k 65536 + j) + i is word i of the Philox block
with counter (k, 0, j, 0), k carrying into the second counter word. (That
ordering was read off the library's output, and the first block for seed 0 is
the generator's well-known first output.)

The oracle keys a particle's stream by (particle id, seed) and counts its
events in the first counter word: event e of particle id is the cuRAND block
at offset 4 * 65536 * e for seed id + 2^32 seed.
"""
import ctypes

import numpy as np
import pytest
from scipy import stats

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
SUBSEQ = 65536


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def curand_stream(seed64: int, offset_words: int, n: int) -> np.ndarray:
    L = _curand()
    gen = ctypes.c_void_p()
    if L.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed64)) == 0
        assert L.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset_words)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out


def curand_block(key, ctr0: int, ctr2: int = 0) -> np.ndarray:
    """Philox block with counter (ctr0 mod 2^32, ctr0 div 2^32, ctr2, 0) from cuRAND."""
    return curand_stream(key[0] + (key[1] << 32), 4 * (ctr0 * SUBSEQ + ctr2), 4)


@pytest.mark.parametrize("pid,seed", [(0, 0), (1, 0), (12345, 0), (0, 1), (4096, 7),
                                      (0xFFFFFFFF, 0xFFFFFFFF), (999_999, 2024)])
def test_philox_matches_curand_events(pid, seed):
    for ev in (0, 1, 2, 3, 17):
        got = oracle.philox([ev, 0, 0, 0], [pid, seed])
        np.testing.assert_array_equal(got, curand_block((pid, seed), ev))


@pytest.mark.parametrize("ctr2", [1, 2, 4095, 65535])
def test_philox_third_counter_word_matches_curand(ctr2):
    for ev in (0, 5):
        got = oracle.philox([ev, 0, ctr2, 0], [42, 9])
        np.testing.assert_array_equal(got, curand_block((42, 9), ev, ctr2))


@pytest.mark.parametrize("event", [1000, 2**20 + 3, 2**31 + 17, 2**32 - 1, 2**32, 2**33 + 5])
def test_philox_large_counters_match_curand(event):
    ctr = [event & 0xFFFFFFFF, event >> 32, 0, 0]
    np.testing.assert_array_equal(oracle.philox(ctr, [77, 3]), curand_block((77, 3), event))


def test_u53_range_and_endpoints():
    assert oracle.u53(0, 0) == 2.0**-53
    assert oracle.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    # 27 high bits of the first word, 26 of the second
    assert oracle.u53(1 << 5, 0) == (2.0**26 + 1) * 2.0**-53
    assert oracle.u53(0, 1 << 6) == 2.0 * 2.0**-53


def test_u53_uniform_ks():
    vals = []
    for ev in range(4000):
        w = oracle.philox([ev, 0, 0, 0], [5, 0])
        vals.append(oracle.u53(w[0], w[1]))
        vals.append(oracle.u53(w[2], w[3]))
    assert stats.kstest(vals, "uniform").pvalue > 1e-3
