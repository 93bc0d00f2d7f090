"""Pins of the oracle's energy, move, refresh and dynamics to facts the paper
and the mathematics fix (not to the oracle itself).

Energy (Eq. Hamiltonian): ferromagnet and gauge-transformed ferromagnet ground
states, exact moments of the density of states, enumeration by two methods.
Move (Eq. Creutz, Eq. flip-OK): the dH value set of Sec. 2.4, the capacity
edge cases, exact conservation of H_EA + H_aux between refreshes, reversibility
(Sec. 2.3). Refresh (Eq. prob-daemons-walkers, Eq. daemons-temperature): exact
cut points at x = 1/2, chi-square and mean. Dynamics: exact invariance of the
canonical measure under one sweep with fresh daemons (Sec. 2.3: detailed
balance), and long-run averages against exact enumeration.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
O = oracle.Oracle()


def neighbours(L):
    """Independent neighbour table (numpy index arithmetic, not the oracle's)."""
    idx = np.arange(L ** 3).reshape(L, L, L)  # [z, y, x]
    fwd = [np.roll(idx, -1, axis=2), np.roll(idx, -1, axis=1), np.roll(idx, -1, axis=0)]
    return [f.reshape(-1) for f in fwd]


def paper_daemon_probs(T):
    """Eq. (prob-daemons-walkers)."""
    b = 1.0 / T
    return np.array([math.exp(-4 * m * b) * (1 - math.exp(-4 * b)) / (1 - math.exp(-16 * b))
                     for m in range(4)])


def paper_daemon_mean(T):
    """Eq. (daemons-temperature): <H_aux>/(gamma N)."""
    b = 1.0 / T
    return 4 * math.exp(-4 * b) / (1 - math.exp(-4 * b)) - 16 * math.exp(-16 * b) / (1 - math.exp(-16 * b))


# ----------------------------------------------------------------- energy --

@pytest.mark.parametrize("L", [2, 3, 4, 5, 6])
def test_ferromagnet_ground_state(L):
    N = L ** 3
    J = np.ones((N, 3), np.int8)
    s = np.ones(N, np.int8)
    assert O.energy(L, J, s) == -3 * N
    s[0] = -1  # one defect breaks its 6 bonds (L > 2) or its 6 bond-slots (L = 2)
    assert O.energy(L, J, s) == -3 * N + 12


@pytest.mark.parametrize("L", [2, 3, 4, 7])
def test_gauge_ferromagnet_ground_state(L):
    """J_xy = eps_x eps_y makes s = eps a state with every bond satisfied."""
    rng = np.random.default_rng(L)
    N = L ** 3
    eps = rng.choice(np.array([-1, 1], np.int8), N)
    nb = neighbours(L)
    J = np.stack([eps * eps[nb[d]] for d in range(3)], axis=1).astype(np.int8)
    assert O.energy(L, J, eps) == -3 * N
    # gauge invariance on random states: H(J^eps, s eps) = H(J, s)
    J0 = O.couplings(L, 99)
    Jg = np.stack([J0[:, d] * eps * eps[nb[d]] for d in range(3)], axis=1).astype(np.int8)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), N)
        assert O.energy(L, Jg, (s * eps).astype(np.int8)) == O.energy(L, J0, s)


def test_dos_exact_moments_l3():
    """Over all 2^N states each bond term averages 0 and the terms are pairwise
    uncorrelated, so sum_E g(E) = 2^N, sum E g(E) = 0, sum E^2 g(E) = 3N 2^N."""
    L, N = 3, 27
    J = O.couplings(L, 3)
    g = O.dos(L, J)
    E = np.arange(-3 * N, 3 * N + 1)
    assert g.sum() == 2 ** N
    assert int((g * E).sum()) == 0
    assert int((g * E * E).sum()) == 3 * N * 2 ** N


def test_dos_two_methods_l2():
    L = 2
    for seed in range(4):
        J = O.couplings(L, seed)
        E = O.all_energies(L, J)
        g = O.dos(L, J)
        hist = np.bincount(E + 24, minlength=49)
        np.testing.assert_array_equal(g, hist)


def test_delta_h_value_set_and_consistency():
    allowed = set(int(v) for v in np.loadtxt(os.path.join(GOLDEN, "delta_h_values.txt")))
    for L in (2, 3, 4, 6):
        J = O.couplings(L, 11 + L)
        s = O.spins(L, 5, L)
        H0 = O.energy(L, J, s)
        for site in range(L ** 3):
            dH = O.delta_h(L, J, s, site)
            assert dH in allowed
            s2 = s.copy()
            s2[site] = -s2[site]
            assert O.energy(L, J, s2) - H0 == dH


# ------------------------------------------------------------------- move --

def _single_site_case(dH_target, m0):
    """Ferromagnetic L = 4 lattice; the site 0 spin pointing along (dH = +12)
    or against (dH = -12) all its neighbours."""
    L = 4
    N = L ** 3
    J = np.ones((N, 3), np.int8)
    s = np.ones(N, np.int8)
    if dH_target == -12:
        s[0] = -1
    m = np.zeros(N, np.uint8)
    m[0] = m0
    assert O.delta_h(L, J, s, 0) == dH_target
    O.half_sweep(L, J, s, m, 0)  # site 0 is even
    return int(s[0]), int(m[0])


def test_capacity_edges_eq_flip_ok():
    # dH = +12: legal only if n = 12 (m = 3) -> n' = 0
    assert _single_site_case(12, 3) == (-1, 0)
    assert _single_site_case(12, 2) == (1, 2)
    # dH = -12: legal only if n = 0 -> n' = 12 (m = 3); m = 1 would need n' = 16
    assert _single_site_case(-12, 0) == (1, 3)
    assert _single_site_case(-12, 1) == (-1, 1)


def test_zero_cost_flip_always_accepted():
    L = 4
    N = L ** 3
    J = np.ones((N, 3), np.int8)
    s = np.ones(N, np.int8)
    # make site 0 have 3 satisfied and 3 unsatisfied bonds: flip its +x, +y, +z neighbours
    nb = neighbours(L)
    for d in range(3):
        s[nb[d][0]] = -1
    for m0 in range(4):
        m = np.zeros(N, np.uint8)
        m[0] = m0
        s2 = s.copy()
        assert O.delta_h(L, J, s2, 0) == 0
        O.half_sweep(L, J, s2, m, 0)
        assert s2[0] == -s[0] and m[0] == m0


@pytest.mark.parametrize("L", [2, 4, 6])
def test_half_sweep_is_an_involution(L):
    """Sec. 2.3: the move undoes itself when repeated with the rest fixed."""
    rng = np.random.default_rng(L)
    N = L ** 3
    J = O.couplings(L, 1)
    for parity in (0, 1):
        for _ in range(5):
            s = rng.choice(np.array([-1, 1], np.int8), N)
            m = rng.integers(0, 4, N).astype(np.uint8)
            s1, m1 = s.copy(), m.copy()
            O.half_sweep(L, J, s1, m1, parity)
            O.half_sweep(L, J, s1, m1, parity)
            np.testing.assert_array_equal(s1, s)
            np.testing.assert_array_equal(m1, m)


@pytest.mark.parametrize("L,serial", [(4, False), (6, False), (3, True), (5, True)])
def test_total_energy_conserved_between_refreshes(L, serial):
    st = O.create(L, 2, 2, 17)
    interval = 1000  # only the refresh at t = 0 happens
    totals = None
    for k in range(40):
        O.run(st, [1.3], interval, serial=serial)
        e, a, _ = O.measure(st)
        if totals is None:
            totals = e + a
        np.testing.assert_array_equal(e + a, totals)


# ---------------------------------------------------------------- refresh --

def test_daemon_cut_points_exact_case():
    rows = np.loadtxt(os.path.join(GOLDEN, "daemon_probs_x_half.txt"))
    T = 4.0 / math.log(2.0)
    th = O.daemon_thresholds(T)
    cum = np.cumsum(rows[:, 1] / rows[:, 2])[:3]
    for k in range(3):
        assert abs(int(th[k]) - cum[k] * 2 ** 32) <= 2


@pytest.mark.parametrize("T", [0.3, 0.7, 1.1, 2.0, 5.0])
def test_refresh_distribution(T):
    L = 32
    counts = np.zeros(4)
    for t in range(0, 40, 10):
        m = O.refresh(L, 1234, 3, t, T)
        counts += np.bincount(m, minlength=4)
    n = counts.sum()
    p = paper_daemon_probs(T)
    expected = n * p
    mask = expected > 5
    chi2 = (((counts - expected) ** 2 / expected)[mask]).sum()
    dof = mask.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * max(dof, 1)) + 10
    mean_n = 4 * (counts * np.arange(4)).sum() / n
    var_n = 16 * (p * np.arange(4) ** 2).sum() - (4 * (p * np.arange(4)).sum()) ** 2
    assert abs(mean_n - paper_daemon_mean(T)) < 5 * math.sqrt(var_n / n) + 1e-12


def test_refresh_limits():
    # beta -> 0: all four values equally likely; beta -> inf: m = 0 always
    th = O.daemon_thresholds(1e300)
    assert [int(v) for v in th] == [2 ** 30, 2 ** 31, 3 * 2 ** 30]
    th = O.daemon_thresholds(1e-3)
    assert [int(v) for v in th] == [2 ** 32] * 3
    with pytest.raises(ValueError):
        O.daemon_thresholds(0.0)
    with pytest.raises(ValueError):
        O.daemon_thresholds(float("nan"))


def test_metro_cut_points():
    for T in (0.5, 1.0, 3.0):
        th = O.metro_thresholds(T)
        for k in range(3):
            assert abs(int(th[k]) - math.exp(-4 * (k + 1) / T) * 2 ** 32) <= 1
    # the extremes: exp(-beta dH) rounds to 1 (every move accepted) once beta dH
    # is below 2^-53, and e^-40 2^32, e^-80/3 2^32 are below 1 (never accepted)
    assert [int(v) for v in O.metro_thresholds(1e20)] == [2 ** 32] * 3
    assert [int(v) for v in O.metro_thresholds(1e6)] == [math.floor(math.exp(-4 * k * 1e-6) * 2 ** 32) for k in (1, 2, 3)]
    assert [int(v) for v in O.metro_thresholds(0.3)] == [math.floor(math.exp(-4 / 0.3) * 2 ** 32), 0, 0]
    assert int(O.metro_thresholds(0.5)[2]) == 0 < int(O.metro_thresholds(0.5)[1])


# --------------------------------------------------- exact L = 2 dynamics --

def _boltzmann(E, T):
    w = np.exp(-(E - E.min()) / T)
    return w / w.sum()


@pytest.mark.parametrize("seed,T", [(0, 0.7), (1, 1.5), (2, 3.0), (3, 10.0)])
def test_micsa_sweep_leaves_canonical_measure_invariant(seed, T):
    """With every daemon drawn from Eq. (prob-daemons-walkers) before the sweep,
    the joint canonical weight is invariant (Sec. 2.3), so pi P = pi exactly."""
    J = O.couplings(2, seed)
    E = O.all_energies(2, J).astype(np.float64)
    pi = _boltzmann(E, T)
    P = O.l2_transition_micsa(J, paper_daemon_probs(T))
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-12)
    # the test has power: the canonical measure at another temperature is not invariant
    pi_wrong = _boltzmann(E, 2.0 * T)
    assert np.abs(pi_wrong @ P - pi_wrong).max() > 1e-4


@pytest.mark.parametrize("seed,T", [(0, 0.7), (5, 2.0)])
def test_metropolis_sweep_leaves_canonical_measure_invariant(seed, T):
    J = O.couplings(2, seed)
    E = O.all_energies(2, J).astype(np.float64)
    pi = _boltzmann(E, T)
    P = O.l2_transition_metro(J, T)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(pi @ P, pi, atol=1e-8)  # cut points quantised to 2^-32


# -------------------------------------------------- long-run statistics --

def _exact_mean_energy(g, N, T):
    E = np.arange(-3 * N, 3 * N + 1, dtype=np.float64)
    w = g * np.exp(-(E - E[g > 0].min()) / T)
    return (w * E).sum() / w.sum() / N


def _batch_mean(x, nb=20):
    x = np.asarray(x, np.float64)
    b = x[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


@pytest.mark.parametrize("L,serial,T,runner", [
    (2, False, 2.0, "micsa"), (2, False, 4.0, "micsa"),
    (3, True, 2.5, "micsa"), (3, True, 5.0, "micsa"),
    (2, False, 2.0, "metro"), (3, True, 3.0, "metro"),
])
def test_long_run_mean_energy_matches_enumeration(L, serial, T, runner):
    N = L ** 3
    st = O.create(L, 1, 1, 1000 + L)
    exact = _exact_mean_energy(O.dos(L, st["J"][0]), N, T)
    chunk = 50
    es = []
    for k in range(800):
        if runner == "micsa":
            O.run(st, np.full(chunk, T), 10, serial=serial)
        else:
            O.run_metropolis(st, np.full(chunk, T), serial=serial)
        if k >= 20:
            es.append(O.measure(st)[0][0] / N)
    mean, err = _batch_mean(es)
    assert abs(mean - exact) < 5 * err + 1e-3, (mean, err, exact)


def test_anneal_reaches_ground_state_l3():
    L, N = 3, 27
    hits = 0
    for seed in range(5):
        st = O.create(L, 1, 1, 500 + seed)
        gs = int(np.nonzero(O.dos(L, st["J"][0]))[0][0]) - 3 * N
        O.run(st, np.linspace(3.0, 0.1, 4000), 5, serial=True)
        hits += int(O.measure(st)[0][0] == gs)
    assert hits >= 4


def test_chunked_run_equals_single_run():
    sched = np.linspace(2.5, 0.5, 137)
    a = O.create(6, 2, 3, 77)
    b = O.create(6, 2, 3, 77)
    O.run(a, sched, 7)
    O.run(b, sched[:50], 7)
    O.run(b, sched[50:51], 7)
    O.run(b, sched[51:], 7)
    assert a["t"] == b["t"] == 137
    np.testing.assert_array_equal(a["s"], b["s"])
    np.testing.assert_array_equal(a["m"], b["m"])


def test_log_refresh_times():
    """Sec. 2.8 procedure: fresh daemons before t = 0, 1, 3, 7, ...; the total
    energy is conserved on every other sweep."""
    st = O.create(6, 1, 1, 31)
    prev = None
    changed_at = []
    for t in range(40):
        O.run_logrefresh(st, [0.9])
        e, a, _ = O.measure(st)
        tot = int(e[0] + a[0])
        if prev is not None and tot != prev:
            changed_at.append(t)
        prev = tot
    assert set(changed_at) <= {1, 3, 7, 15, 31}
    assert len(changed_at) >= 3


# ------------------------------------------------ planted mistakes fail --

def test_planted_capacity_mistake_is_caught():
    bad = oracle.Oracle(mutant=1)
    J = np.ones((64, 3), np.int8)
    s = np.ones(64, np.int8)
    s[0] = -1
    m = np.zeros(64, np.uint8)
    m[0] = 1
    bad.half_sweep(4, J, s, m, 0)
    assert (int(s[0]), int(m[0])) != (-1, 1)


def test_planted_sign_mistake_breaks_conservation():
    bad = oracle.Oracle(mutant=2)
    st = bad.create(4, 1, 1, 17)
    bad.run(st, [1.3], 1000)
    e0, a0, _ = bad.measure(st)
    bad.run(st, [1.3], 1000)
    e1, a1, _ = bad.measure(st)
    assert int(e0[0] + a0[0]) != int(e1[0] + a1[0])


def test_planted_bond_mistake_breaks_delta_h():
    bad = oracle.Oracle(mutant=3)
    L = 4
    J = bad.couplings(L, 15)
    s = bad.spins(L, 5, 4)
    H0 = bad.energy(L, J, s)
    mismatch = 0
    for site in range(L ** 3):
        s2 = s.copy()
        s2[site] = -s2[site]
        mismatch += bad.energy(L, J, s2) - H0 != bad.delta_h(L, J, s, site)
    assert mismatch > 0


def test_planted_refresh_mistake_breaks_distribution():
    bad = oracle.Oracle(mutant=4)
    T = 2.0
    m = bad.refresh(32, 1234, 3, 0, T)
    counts = np.bincount(m, minlength=4)
    expected = counts.sum() * paper_daemon_probs(T)
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 > 100


# ------------------------------------------- gamma daemons and walkers --

def test_run_ex_reduces_to_gamma_one():
    sched = np.linspace(2.5, 0.5, 45)
    a = O.create(6, 2, 2, 41)
    b = O.create(6, 2, 2, 41, gamma=1, walkers=False)
    O.run(a, sched, 7)
    O.run_ex(b, sched, 7)
    np.testing.assert_array_equal(a["s"], b["s"])
    np.testing.assert_array_equal(a["m"], b["m"])
    c = O.create(6, 1, 2, 42)
    d = O.create(6, 1, 2, 42)
    O.run_logrefresh(c, sched)
    O.run_ex(d, sched, 0)
    np.testing.assert_array_equal(c["s"], d["s"])
    np.testing.assert_array_equal(c["m"], d["m"])


@pytest.mark.parametrize("direction", range(6))
def test_wandering_cycle_moves_walkers_two_sites(direction):
    """Sec. 2.6: in a two-timestep cycle the even sites, then the odd sites,
    exchange their walker with the neighbour along the direction. A walker that
    starts on an even site ends two sites on along the direction, one that
    starts on an odd site two sites back; after L/2 cycles (L timesteps) every
    walker is back where it started."""
    L = 6
    rng = np.random.default_rng(direction)
    m0 = rng.integers(0, 4, L ** 3).astype(np.uint8)
    m = m0.copy()
    O.wander(L, m, direction, 0)
    O.wander(L, m, direction, 1)
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    even = ((x + y + z) % 2 == 0).reshape(-1)
    step = np.zeros(3, int)
    step[direction % 3] = 1 if direction < 3 else -1  # (dx, dy, dz)
    expect = np.zeros_like(m0)
    for site in range(L ** 3):
        sz, sy, sx = np.unravel_index(site, (L, L, L))
        k = 2 if even[site] else -2
        tx, ty, tz = (sx + k * step[0]) % L, (sy + k * step[1]) % L, (sz + k * step[2]) % L
        expect[(tz * L + ty) * L + tx] = m0[site]
    np.testing.assert_array_equal(m, expect)
    for _ in range(L // 2 - 1):
        O.wander(L, m, direction, 0)
        O.wander(L, m, direction, 1)
    np.testing.assert_array_equal(m, m0)


@pytest.mark.parametrize("gamma,walkers", [(3, False), (2, True), (6, True)])
def test_total_energy_conserved_with_gamma_and_walkers(gamma, walkers):
    st = O.create(4, 1, 2, 23, gamma=gamma, walkers=walkers)
    totals = None
    for _ in range(25):
        O.run_ex(st, [1.2], 1000)
        e, a, _ = O.measure(st)
        if totals is None:
            totals = e + a
        np.testing.assert_array_equal(e + a, totals)


@pytest.mark.parametrize("gamma,walkers", [(2, False), (1, True), (6, True)])
def test_long_run_gamma_walkers_match_enumeration(gamma, walkers):
    """Refreshes and sweeps leave the canonical measure of spins and all gamma
    daemons invariant, and wandering only permutes daemons, so long-run averages
    are canonical."""
    L, N, T = 2, 8, 2.0
    st = O.create(L, 1, 1, 900 + gamma, gamma=gamma, walkers=walkers)
    exact = _exact_mean_energy(O.dos(L, st["J"][0]), N, T)
    es = []
    for k in range(600):
        O.run_ex(st, np.full(40, T), 10)
        if k >= 20:
            es.append(O.measure(st)[0][0] / N)
    mean, err = _batch_mean(es)
    assert abs(mean - exact) < 5 * err + 1e-3, (mean, err, exact)


# ------------------------------------------------ four-point correlation --

def test_correlation_matches_fft_autocorrelation():
    """C4 of Sec. 3 is a circular autocorrelation of the overlap field q along
    each axis; numpy's FFT computes it independently."""
    L, S, R = 6, 2, 3
    st = O.create(L, S, R, 61)
    O.run(st, np.linspace(2.0, 1.0, 15), 4)
    G = O.correlation(st)
    for a in range(S):
        ref = np.zeros(L)
        for ra in range(R):
            for rb in range(ra + 1, R):
                q = (st["s"][a, ra].astype(np.int64) * st["s"][a, rb]).reshape(L, L, L)
                for axis in range(3):
                    f = np.fft.fft(q, axis=axis)
                    ac = np.fft.ifft(f * np.conj(f), axis=axis).real  # sum_x q_x q_{x + r}
                    ref += np.moveaxis(ac, axis, 0).reshape(L, -1).sum(axis=1)
        np.testing.assert_array_equal(G[a], np.rint(ref).astype(np.int64))
    npairs = R * (R - 1) // 2
    np.testing.assert_array_equal(G[:, 0], 3 * L ** 3 * npairs)  # C4(0) = 1


def test_correlation_identical_replicas_is_one():
    L = 4
    st = O.create(L, 1, 2, 5)
    st["s"][0, 1] = st["s"][0, 0]
    np.testing.assert_array_equal(O.correlation(st)[0], 3 * L ** 3)


def acceptance_z_scores(orc, L=16, T=3.0, seed=41, refreshes=60):
    """Per dE class over the even sites of an L lattice and `refreshes` fresh daemon
    draws: (accepted fraction - closed form) / standard error, and the class counts."""
    x = np.exp(-4.0 / T)
    J = orc.couplings(L, seed)
    s = orc.spins(L, seed, 0)
    sites = np.arange(L ** 3)
    xs, ys, zs = sites % L, (sites // L) % L, sites // (L * L)
    even = sites[(xs + ys + zs) % 2 == 0]
    acc, tot = {}, {}
    for t in range(refreshes):
        m = orc.refresh(L, seed, 0, t, T)
        dE = np.array([orc.delta_h(L, J, s, int(i)) for i in even])
        s_new, m_new = s.copy(), m.copy()
        orc.half_sweep(L, J, s_new, m_new, 0)
        flipped = s_new[even] != s[even]
        for d in np.unique(dE):
            sel = dE == d
            acc[d] = acc.get(d, 0) + int(flipped[sel].sum())
            tot[d] = tot.get(d, 0) + int(sel.sum())
        orc.half_sweep(L, J, s_new, m_new, 1)  # move the odd sites too: new local fields
        s = s_new
    z = {}
    for d in sorted(tot):
        j = abs(d) // 4
        p = (x ** j - x ** 4) / (1 - x ** 4) if d > 0 else (1 - x ** (4 - j)) / (1 - x ** 4)
        se = np.sqrt(max(p * (1 - p), 1e-12) / tot[d])
        z[d] = (acc[d] / tot[d] - p) / se
    return z, tot


def test_acceptance_with_fresh_daemons_follows_the_truncated_geometric_law():
    """With the daemons drawn fresh before a half-sweep, p(m) = x^m / (1 + x + x^2 + x^3),
    x = exp(-4/T), m = 0..3 (Eq. (prob-daemons-walkers)), and Eq. (flip-OK): a flip that
    costs dE = 4j > 0 is accepted iff m >= j, with probability (x^j - x^4) / (1 - x^4);
    one that gains dE = -4j <= 0 iff the daemon can hold the surplus, m <= 3 - j, with
    probability (1 - x^(4 - j)) / (1 - x^4). Frequencies per dE class over the even
    sites of an L = 16 lattice and 60 refreshes agree within 5 standard errors."""
    z, tot = acceptance_z_scores(O)
    assert set(tot) == {-12, -8, -4, 0, 4, 8, 12}
    assert min(tot.values()) > 100  # every class is sampled
    assert max(abs(v) for v in z.values()) <= 5.0, z


@pytest.mark.parametrize("mutant", [1, 2, 4])
def test_planted_mistakes_break_the_acceptance_law(mutant):
    # capacity one step too large, the daemon absorbing the wrong sign, a wrong
    # Boltzmann factor in the refresh: each moves some class far outside 5 errors
    z, _ = acceptance_z_scores(oracle.Oracle(mutant=mutant))
    assert max(abs(v) for v in z.values()) > 10.0, z
