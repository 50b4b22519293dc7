"""Pin the oracle's Philox4x32-10 to an implementation it shares nothing
with: cuRAND's host-side PHILOX4_32_10 generator (a library run on the CPU).

cuRAND's host generator lays its output out so that 128-bit block b is
Philox4x32-10 of counter (b // 65536 as a 64-bit pair in words 0-1,
b % 65536 in word 2, 0 in word 3) under key (seed lo, seed hi).  That layout
was established by experiment; the test checks it block by block, so a wrong
round function, key schedule, multiplier, Weyl constant, or counter/key word
placement in the oracle fails here.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not os.path.isabs(c)):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    pytest.skip("libcurand not available")


def _curand_blocks(seed, offset_blocks, n_blocks):
    lib = _curand()
    g = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(g), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * offset_blocks)) == 0
        buf = (ctypes.c_uint * (4 * n_blocks))()
        assert lib.curandGenerate(g, buf, 4 * n_blocks) == 0
        return np.frombuffer(buf, dtype=np.uint32).reshape(n_blocks, 4).copy()
    finally:
        lib.curandDestroyGenerator(g)


def _counter(b):
    hi = b // 65536
    return [hi & 0xFFFFFFFF, hi >> 32, b % 65536, 0]


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
@pytest.mark.parametrize("offset", [0, 65536 * 7 + 11, (1 << 40) + 65535, (1 << 52) + 3])
def test_philox_matches_curand_host(seed, offset):
    blocks = _curand_blocks(seed, offset, 3)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(3):
        b = offset + i
        got = oracle.philox4x32_10(_counter(b), key)
        assert list(got) == list(blocks[i]), (seed, b)


def test_philox_first_block_zero_key_zero_counter():
    # the all-zero input, from the cuRAND host generator with seed 0
    blocks = _curand_blocks(0, 0, 1)
    assert list(oracle.philox4x32_10([0, 0, 0, 0], [0, 0])) == list(blocks[0])
