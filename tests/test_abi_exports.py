"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
declared in include/*.h, and its host-only cut-point functions agree exactly
with the oracle's (both compute them independently in IEEE double)."""
import glob
import math
import os
import re

import numpy as np
import pytest

import oracle
import paper_2506_16240_gb300 as micsa
from paper_2506_16240_gb300 import build as micsa_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(micsa_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    micsa_build.build()
    return micsa.lib()


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 16
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert names <= set(micsa.SIGNATURES), "binding lacks a declared entry point"


def test_daemon_cut_points_match_oracle_exactly(lib):
    O = oracle.Oracle()
    Ts = [1e-3, 0.05, 0.3, 0.5, 0.7, 1.0, 1.1019, 1.4, 2.0, 2.5, 3.0, 5.0, 1e3, 1e300,
          4.0 / math.log(2.0)]
    Ts += list(np.linspace(0.1, 6.0, 500))
    for T in Ts:
        np.testing.assert_array_equal(micsa.daemon_thresholds(T), O.daemon_thresholds(T),
                                      err_msg=f"T={T}")
        np.testing.assert_array_equal(micsa.metro_thresholds(T), O.metro_thresholds(T),
                                      err_msg=f"T={T}")


def test_bad_temperatures_rejected(lib):
    for T in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(micsa.MicsaError):
            micsa.daemon_thresholds(T)
        with pytest.raises(micsa.MicsaError):
            micsa.metro_thresholds(T)


def test_pool_job_bytes_counts_plane_storage_for_plane_jobs(lib):
    """Host-only: a job's arena bytes are its bonds, spins, daemons, best
    configuration and refresh cut points, plus bit-plane storage exactly for the
    jobs the pool sweeps as bit planes (even L above 32)."""
    def align(n):
        return (n + 255) // 256 * 256

    for L in (8, 16, 30, 32, 34, 40, 42, 48, 50, 64, 66, 72, 96, 128):
        for R, n, r in ((1, 1000, 10), (2, 77, 5), (4, 10, 1)):
            Lh = L // 2
            P = 4 * ((Lh + 3) // 4)
            half = L * L * P
            n_refresh = max(1, (n + r - 1) // r)
            expect = align(2 * half) + 2 * align(R * 2 * half) + align(R * max(L ** 3, 2 * half)) + align(24 * n_refresh)
            WP = L * ((L + 31) // 32) * P  # rows of P plane words
            if L % 2 == 0 and L > 32:
                expect += align(4 * 6 * WP * R) + align(4 * 12 * WP)
            elif L <= 32:  # bond planes only (the shared-memory path of small lattices)
                expect += align(4 * 12 * WP)
            assert micsa.Pool.job_bytes(L, R, n, r) == expect, (L, R, n, r)


def test_pool_calls_reject_a_null_pool(lib):
    assert lib.micsa_pool_set_planes(None, 1) == micsa.MICSA_E_INVALID_ARG
    assert lib.micsa_pool_set_shape(None, 4, 2) == micsa.MICSA_E_INVALID_ARG
    assert lib.micsa_pool_set_launch_config(None, 0, 1, 1) == micsa.MICSA_E_INVALID_ARG
