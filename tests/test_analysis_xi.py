"""Integral estimators of the four-point correlation, I_n and xi_{n,n+1} =
I_{n+1} / I_n (Sec. 3, Eq. (xi-def)), pinned to closed forms of the lattice sums."""
import numpy as np
import pytest

from paper_2506_16240_gb300 import analysis


def periodic(f, L):
    r = np.arange(L)
    return f(np.minimum(r, L - r))


@pytest.mark.parametrize("q", [0.3, 0.6, 0.8])
def test_exponential_correlation_gives_the_geometric_series_lengths(q):
    # sum r q^r = q/(1-q)^2, sum r^2 q^r = q(1+q)/(1-q)^3, sum r^3 q^r = q(1+4q+q^2)/(1-q)^4
    L = 512  # q^(L/2) is negligible: the truncated sums equal the infinite ones
    c4 = periodic(lambda r: q ** r, L)
    assert analysis.xi(c4, 1) == pytest.approx((1 + q) / (1 - q), rel=1e-12)
    assert analysis.xi(c4, 2) == pytest.approx((1 + 4 * q + q * q) / ((1 - q) * (1 + q)), rel=1e-12)
    I, stop = analysis.c4_integrals(c4, 1)
    assert stop == L // 2
    assert I[0] == pytest.approx(1 / (1 - q), rel=1e-12) and I[1] == pytest.approx(q / (1 - q) ** 2, rel=1e-12)


def test_constant_correlation_gives_power_sums_to_half_the_lattice():
    # identical replicas: C4 = 1 at every distance
    L = 40
    I, stop = analysis.c4_integrals(np.ones(L), 3)
    m = L // 2
    assert stop == m
    assert list(I) == [m + 1, m * (m + 1) / 2, m * (m + 1) * (2 * m + 1) / 6, (m * (m + 1) / 2) ** 2]
    assert analysis.xi(np.ones(L)) == pytest.approx((2 * m + 1) / 3)


def test_sum_stops_before_the_first_non_positive_value():
    c4 = np.array([1.0, 0.5, 0.25, -0.01, 0.2, 0.1, 0.0, 0.1])  # L = 8: r = 0..4 considered
    I, stop = analysis.c4_integrals(c4, 2)
    assert stop == 2
    assert I[1] == pytest.approx(0.5 + 2 * 0.25) and I[2] == pytest.approx(0.5 + 4 * 0.25)
    assert analysis.xi(c4) == pytest.approx(1.5 / 1.0)


def test_sum_stops_where_the_signal_falls_below_its_noise():
    c4 = np.array([1.0, 0.5, 0.2, 0.05, 0.04, 0.03, 0.02, 0.01, 0.0, 0.01])  # L = 10: r = 0..5
    err = np.full(10, 0.02)  # 3 sigma = 0.06: r = 3 (0.05) is noise
    I, stop = analysis.c4_integrals(c4, 2, err)
    assert stop == 2 and I[2] == pytest.approx(0.5 + 4 * 0.2)
    assert analysis.c4_integrals(c4, 2)[1] == 5  # without errors: every positive value counts


def test_sample_average_uses_the_standard_error_of_the_mean():
    rng = np.random.default_rng(0)
    L, S, q = 64, 16, 0.5
    base = periodic(lambda r: q ** r, L)
    samples = base + rng.normal(0.0, 1e-3, (S, L))  # noise far below the signal at small r
    # the tail is cut where q^r falls below three standard errors (1e-3 / 4 each): near r = 10;
    # up to that point the estimate equals the noiseless truncated sums
    mean = samples.mean(axis=0)
    err = samples.std(axis=0, ddof=1) / np.sqrt(S)
    I, stop = analysis.c4_integrals(mean, 2, err)
    assert 8 <= stop <= 12
    r = np.arange(stop + 1)
    exact = np.sum(r ** 2 * q ** r) / np.sum(r * q ** r)
    assert analysis.xi_of_samples(samples) == pytest.approx(exact, rel=1e-2)  # noise of the last terms
    # one sample: no error estimate, the positive-value rule alone (the sum runs to L/2)
    r = np.arange(L // 2 + 1)
    assert analysis.xi_of_samples(base[None, :]) == pytest.approx(np.sum(r ** 2 * q ** r) / np.sum(r * q ** r),
                                                                  rel=1e-12)
