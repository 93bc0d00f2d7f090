"""Pins of the oracle's initial data and of its replica overlap.

Couplings (Sec. 2.1, Eq. Hamiltonian): every bond is J = +-1 with probability
1/2, drawn independently of every other bond. Checked by the mean of each bond
direction, the correlations between the three bonds of one site, between
neighbouring sites and between samples (each within 5 standard errors of 0 on
L = 32), and by rebuilding J from cuRAND's host Philox4x32-10 generator with the
counter layout stated in the oracle's header.

Spins (Sec. 3, the fully disordered infinite-temperature start): s = +-1 with
probability 1/2, independent across sites and replicas. Checked by the
magnetisation, the neighbour correlation and the overlap of two replicas (within
5 standard errors of 0), and by the same library rebuild.

Overlap (Sec. 3 and App. C, q^{ab} = sum_x s^a_x s^b_x over replica pairs a < b):
against numpy's einsum on random states, identical replicas give N and a
replica flipped everywhere gives -N.

Each pin fails on the planted mistake it guards (-DORC_MUTANT=5, 6, 7).
"""
import itertools

import numpy as np
import pytest

import oracle
from curand_host import curand, philox_blocks

O = oracle.Oracle()


def _z(mean, n):
    """z-score of the mean of n independent +-1 values of expectation 0."""
    return mean * np.sqrt(n)


def coupling_z_scores(orc, L=32, samples=4, seed=2506):
    """z-scores of the statistics that are 0 for fair, independent bonds."""
    J = np.stack([orc.couplings(L, seed, a) for a in range(samples)]).astype(np.int64)  # [S, N, 3]
    n = J.shape[0] * J.shape[1]
    z = {}
    for d in range(3):
        z[f"mean_{d}"] = _z(J[:, :, d].mean(), n)
    for d, e in itertools.combinations(range(3), 2):
        z[f"corr_{d}{e}"] = _z((J[:, :, d] * J[:, :, e]).mean(), n)
    # the +x bond of a site against the +x bond of its +x neighbour
    Jx = J[:, :, 0].reshape(samples, L, L, L)
    z["corr_neighbour"] = _z((Jx * np.roll(Jx, -1, axis=3)).mean(), n)
    # two samples drawn from the same seed
    z["corr_samples"] = _z((J[0] * J[1]).mean(), 3 * J.shape[1])
    return z


def spin_z_scores(orc, L=32, seed=77, gids=(0, 1, 2, 3)):
    s = np.stack([orc.spins(L, seed, g) for g in gids]).astype(np.int64)  # [G, N]
    N = s.shape[1]
    z = {"mean": _z(s.mean(), s.size)}
    sg = s.reshape(len(gids), L, L, L)
    z["corr_neighbour"] = _z((sg * np.roll(sg, -1, axis=3)).mean(), s.size)
    for a, b in itertools.combinations(range(len(gids)), 2):
        z[f"overlap_{a}{b}"] = _z((s[a] * s[b]).mean(), N)
    return z


def overlap_mismatches(orc, L=6, S=3, R=4, seed=5):
    """Count of overlap entries that differ from numpy's einsum on random states,
    plus the results for identical and flipped replicas."""
    rng = np.random.default_rng(seed)
    N = L ** 3
    st = orc.create(L, S, R, 1)
    st["s"] = np.where(rng.random((S, R, N)) < 0.5, 1, -1).astype(np.int8)
    st["m"] = rng.integers(0, 4, (S, R, N)).astype(np.uint8)
    _, aux, q = orc.measure(st)
    ref = [int(np.einsum("i,i->", st["s"][a, ra].astype(np.int64), st["s"][a, rb].astype(np.int64)))
           for a in range(S) for ra, rb in itertools.combinations(range(R), 2)]
    bad = int(np.sum(np.asarray(ref) != q))
    aux_ref = 4 * st["m"].reshape(S * R, N).astype(np.int64).sum(axis=1)
    bad += int(np.sum(aux_ref != aux))
    same = orc.create(L, 1, 2, 1)
    same["s"][0, 1] = same["s"][0, 0]
    flipped = orc.create(L, 1, 2, 1)
    flipped["s"][0, 1] = -flipped["s"][0, 0]
    return bad, int(orc.measure(same)[2][0]), int(orc.measure(flipped)[2][0])


# ------------------------------------------------------------- couplings --

def test_couplings_are_fair_and_independent():
    z = coupling_z_scores(O)
    assert max(abs(v) for v in z.values()) < 5.0, z


def test_couplings_are_plus_minus_one():
    J = O.couplings(8, 3, 0)
    assert set(np.unique(J).tolist()) == {-1, 1}


@pytest.mark.skipif(curand is None, reason="libcurand not found")
@pytest.mark.parametrize("sample", [0, 3])
def test_couplings_rebuilt_from_library_philox(sample):
    """Bond d of site i is -1 iff word d of the Philox block of counter
    (i, 0, 4 * sample + 0, 0) is at least 2^31 (the counter layout of the header)."""
    L, seed = 6, 0x1234_5678_9ABC
    blocks = philox_blocks(seed, range(L ** 3), (sample << 2) | 0)
    ref = np.where(blocks[:, :3] >= 0x80000000, -1, 1).astype(np.int8)
    np.testing.assert_array_equal(O.couplings(L, seed, sample), ref)


# ------------------------------------------------------------------ spins --

def test_initial_spins_are_fair_and_independent():
    z = spin_z_scores(O)
    assert max(abs(v) for v in z.values()) < 5.0, z


@pytest.mark.skipif(curand is None, reason="libcurand not found")
@pytest.mark.parametrize("gid", [0, 5])
def test_initial_spins_rebuilt_from_library_philox(gid):
    """s_i = -1 iff word 0 of the block of counter (i, 0, 4 * gid + 1, 0) is at least 2^31."""
    L, seed = 6, 99
    blocks = philox_blocks(seed, range(L ** 3), (gid << 2) | 1)
    ref = np.where(blocks[:, 0] >= 0x80000000, -1, 1).astype(np.int8)
    np.testing.assert_array_equal(O.spins(L, seed, gid), ref)


# ---------------------------------------------------------------- overlap --

def test_overlap_matches_einsum_and_limits():
    bad, same, flipped = overlap_mismatches(O)
    assert bad == 0
    assert same == 6 ** 3 and flipped == -(6 ** 3)


# ------------------------------------------------ planted mistakes fail --

def test_planted_one_word_for_three_bonds_is_caught():
    z = coupling_z_scores(oracle.Oracle(mutant=5))
    assert max(abs(v) for v in z.values()) > 100, z


def test_planted_biased_spins_are_caught():
    z = spin_z_scores(oracle.Oracle(mutant=6))
    assert abs(z["mean"]) > 100, z


def test_planted_self_overlap_is_caught():
    bad, same, flipped = overlap_mismatches(oracle.Oracle(mutant=7))
    assert bad > 0 or flipped != -(6 ** 3)
