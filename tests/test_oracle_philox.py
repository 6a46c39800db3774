"""Pins of the oracle's Philox-4x32-10 block function and uniform mapping.

cuRAND's host-side Philox generator is an independent implementation of the same
published definition (Salmon et al., SC'11).  It runs on the CPU; its output
block b for seed s is Philox(counter = (q_lo, q_hi, b mod 65536, 0), key = s)
with q = b div 65536.  Matching it over 2^18 blocks, at 64-bit counter offsets
and for several 64-bit seeds pins the multipliers, the Weyl key schedule, the
round count and the output order.  The fourth counter word is pinned on the
GPU against cuRAND's device function (tests/test_gpu_toygen.py).
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest


def _curand():
    for cand in ("/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")):
        if cand and (os.path.exists(cand) or not cand.startswith("/")):
            try:
                return ctypes.CDLL(cand)
            except OSError:
                pass
    pytest.skip("libcurand not available")


def _host_philox(lib, seed, n_blocks, offset_blocks=0):
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:   # CURAND_RNG_PSEUDO_PHILOX4_32_10
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        if offset_blocks:
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        buf = (ctypes.c_uint32 * (4 * n_blocks))()
        assert lib.curandGenerate(gen, buf, 4 * n_blocks) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return np.frombuffer(buf, dtype=np.uint32).astype(np.uint64).reshape(-1, 4)


@pytest.mark.parametrize("seed", [0, 777, 0xDEADBEEFCAFEF00D, 2**64 - 1])
@pytest.mark.parametrize("offset", [0, (1 << 32) * 65536 + 5 * 65536 + 3, 65536 * 7 + 9])
def test_philox_matches_curand_host(oracle, seed, offset):
    lib = _curand()
    n = 1 << 18 if offset == 0 else 4096
    ref = _host_philox(lib, seed, n, offset)
    b = np.arange(n, dtype=np.uint64) + np.uint64(offset)
    q = b // np.uint64(65536)
    out = oracle.philox4x32_10(q & np.uint64(0xFFFFFFFF), q >> np.uint64(32), b % np.uint64(65536),
                               np.zeros(n, np.uint64), seed & 0xFFFFFFFF, seed >> 32)
    np.testing.assert_array_equal(np.stack(out, axis=1), ref)


def test_u01_mapping(oracle):
    assert oracle.u01(0, 0)[()] == 2.0 ** -53
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF)[()] == 1.0
    assert oracle.u01(0x80000000, 0)[()] == 0.5 + 2.0 ** -53
    a = np.arange(1000, dtype=np.uint64) * np.uint64(4294967)
    u = oracle.u01(a, np.zeros_like(a))
    assert np.all(np.diff(u) > 0) and np.all((u > 0) & (u <= 1))
    # exact: the mantissa of u * 2^53 is an integer
    assert np.all(np.floor(u * 2.0 ** 53) == u * 2.0 ** 53)


def test_counter_words_are_distinct_streams(oracle):
    n = 4096
    i = np.arange(n, dtype=np.uint64)
    z = np.zeros(n, np.uint64)
    outs = [np.stack(oracle.philox4x32_10(*(i if w == j else z for w in range(4)), 5, 9), axis=1)
            for j in range(4)]
    allv = np.concatenate([o.ravel() for o in outs])
    assert np.unique(allv).size > 0.999 * allv.size
    # uniformity of the 32-bit words: chi^2 over 16 bins
    hist = np.bincount((allv >> np.uint64(28)).astype(np.int64), minlength=16)
    exp = allv.size / 16
    assert ((hist - exp) ** 2 / exp).sum() < 60
