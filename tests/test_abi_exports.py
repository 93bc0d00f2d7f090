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
