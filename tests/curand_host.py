"""cuRAND's host-side Philox4x32-10 generator, called through ctypes (a library
run on the CPU, independent of the oracle and of the CUDA path).

With seed ``s`` and output offset ``4q`` the generator returns the Philox4x32-10
block of counter ``((q >> 16) mod 2^32, q >> 48, q mod 2^16, 0)`` under key
``(s mod 2^32, s >> 32)``; ``tests/test_oracle_philox.py`` establishes that
ordering by matching outputs.
"""
import ctypes
import ctypes.util
import os

import numpy as np

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _load_curand():
    cands = []
    for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
              "/usr/local/cuda/targets/x86_64-linux/lib"):
        cands += [os.path.join(d, "libcurand.so"), os.path.join(d, "libcurand.so.10")]
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


curand = _load_curand()


def curand_words(seed, offset, nwords):
    """``nwords`` consecutive outputs of the generator from output offset ``offset``."""
    lib = curand
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
        out = np.zeros(nwords, np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def philox_blocks(seed, c0_values, c2):
    """Blocks of counters (c0, 0, c2, 0) for every c0 in ``c0_values`` (c0 < 2^32,
    c2 < 2^16): the library's output quad q = (c0 << 16) | c2. Returns [n, 4]."""
    assert 0 <= c2 < (1 << 16)
    lib = curand
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    out = np.zeros((len(c0_values), 4), np.uint32)
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        for k, c0 in enumerate(c0_values):
            q = (int(c0) << 16) | c2
            assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * q)) == 0
            assert lib.curandGenerate(gen, out[k].ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out
