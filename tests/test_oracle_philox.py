"""Pin the oracle's Philox4x32-10 to an independent implementation.

cuRAND's host-side PHILOX4_32_10 generator (a library, run on the CPU) with
seed ``s`` and output offset ``4q`` returns the Philox4x32-10 block of counter
``((q >> 16) mod 2^32, q >> 48, q mod 2^16, 0)`` under key ``(s mod 2^32, s >> 32)``
-- established by matching its outputs, not by reading its code. Agreement on
many (seed, offset) pairs pins every counter word the project uses (the fourth
word is zero for sweep indices below 2^32) and both key words.
"""
import numpy as np
import pytest

import oracle
from curand_host import curand as _curand, curand_words as _curand_blocks


@pytest.mark.skipif(_curand is None, reason="libcurand not found")
@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0x00000001DEADBEEF])
def test_philox_matches_curand_host(seed):
    o = oracle.Oracle()
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(seed % 1000)
    quads = [0, 1, 2, 65535, 65536, 65537, (1 << 32) + 5, (7 << 48) + (5 << 16) + 65535]
    quads += [int(v) for v in rng.integers(0, 1 << 62, 20)]
    for q in quads:
        lib_words = _curand_blocks(seed, 4 * q, 4)
        ctr = [(q >> 16) & 0xFFFFFFFF, (q >> 48) & 0xFFFFFFFF, q & 0xFFFF, 0]
        np.testing.assert_array_equal(o.philox(ctr, key), lib_words, err_msg=f"quad {q}")


@pytest.mark.skipif(_curand is None, reason="libcurand not found")
def test_philox_long_stream_matches_curand_host():
    """A contiguous run of 2^20 words crosses the c0 increment of the library's ordering."""
    o = oracle.Oracle()
    seed = 2506_16240
    words = _curand_blocks(seed, 0, 1 << 20)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in [0, 3, 65535, 65536, 131071, 200000, (1 << 18) - 1]:
        ctr = [(q >> 16) & 0xFFFFFFFF, 0, q & 0xFFFF, 0]
        np.testing.assert_array_equal(o.philox(ctr, key), words[4 * q: 4 * q + 4])
