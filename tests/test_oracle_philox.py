"""Pin the oracle's Philox-4x32-10 (convention C4) to cuRAND's host generator.

cuRAND's host-side CURAND_RNG_PSEUDO_PHILOX4_32_10 generator runs on the CPU
and is an implementation independent of the oracle. With seed s it emits, for
output block b (4 words), Philox-4x32-10 of counter (b >> 16, 0, b & 0xffff, 0)
under key (s & 0xffffffff, s >> 32); the block order was established by
matching blocks one by one and is itself re-checked by these tests at many
offsets. A wrong multiplier, Weyl increment, round count, word permutation or
key split makes every block differ.
"""
import ctypes
import ctypes.util
import os

import numpy as np
import pytest

import oracle

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", "/usr/local/cuda/lib64/libcurand.so.10",
             ctypes.util.find_library("curand") or ""]
    for c in cands:
        if c and os.path.exists(c):
            try:
                return ctypes.CDLL(c)
            except OSError:
                pass
    pytest.skip("libcurand not found")


def _curand_blocks(seed: int, first_block: int, n_blocks: int) -> np.ndarray:
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * n_blocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(n_blocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 3, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0xDEADBEEF00000000])
def test_philox_matches_curand_host(seed):
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for first in (0, 65530, (7 << 16) + 12345, (0xFFFF << 16) + 65500):
        blocks = _curand_blocks(seed, first, 64)
        for j in range(64):
            b = first + j
            got = oracle.philox((b >> 16, 0, b & 0xFFFF, 0), key)
            assert np.array_equal(got, blocks[j]), (seed, b)


def test_philox_counter_and_key_sensitivity():
    # Every input word reaches every output word: flipping one input bit
    # changes about half of the 128 output bits (avalanche of ten rounds).
    base = oracle.philox((1, 2, 3, 4), (5, 6))
    for word in range(6):
        for bit in (0, 17, 31):
            ctr = [1, 2, 3, 4]
            key = [5, 6]
            if word < 4:
                ctr[word] ^= 1 << bit
            else:
                key[word - 4] ^= 1 << bit
            out = oracle.philox(ctr, key)
            flipped = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, out))
            assert 32 <= flipped <= 96, (word, bit, flipped)
