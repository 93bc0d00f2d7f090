"""Host-side analysis of measured relaxation curves.

The paper compares MicSA with the canonical (Metropolis) dynamics by a single
time-rescaling factor k: after t_plot = k * t_MicSA the two relaxations coincide,
and k* ~ gamma for gamma walkers per spin (Sec. 3, Table (k*), Fig. 1). The
paper extracts k* from the coherence length xi_12 = I_2 / I_1 (Eq. (xi-def)),
with the integrals of C4 estimated as in its references. Here the integrals
are lattice sums cut where C4 falls into its noise (c4_integrals), and the same
fit of k (fit_time_rescaling) applies to xi_12(t) and to the energy per spin,
which the paper also compares after the rescaling (Fig. 1, Eq. (delta1)).
"""
import numpy as np


def rescaled_mismatch(t_ref, e_ref, t, e, k):
    """Mean squared difference between e(t) and the reference curve at k t, the
    reference interpolated linearly in log t; points with k t outside the
    reference range are left out. Returns (mismatch, points used)."""
    t_ref = np.asarray(t_ref, np.float64)
    e_ref = np.asarray(e_ref, np.float64)
    t = np.asarray(t, np.float64)
    e = np.asarray(e, np.float64)
    kt = k * t
    use = (kt >= t_ref[0]) & (kt <= t_ref[-1])
    if not np.any(use):
        return np.inf, 0
    ref = np.interp(np.log(kt[use]), np.log(t_ref), e_ref)
    return float(np.mean((e[use] - ref) ** 2)), int(use.sum())


def fit_time_rescaling(t_ref, e_ref, t, e, k_range=(0.5, 50.0), min_points=4):
    """k minimising rescaled_mismatch over a log-spaced scan of k_range, refined
    by golden-section search around the best scan point. t_ref and t must be
    increasing and positive; returns (k, mismatch, points used)."""
    lo, hi = np.log(k_range[0]), np.log(k_range[1])
    grid = np.exp(np.linspace(lo, hi, 400))

    def f(k):
        m, n = rescaled_mismatch(t_ref, e_ref, t, e, k)
        return m if n >= min_points else np.inf

    vals = np.array([f(k) for k in grid])
    i = int(np.argmin(vals))
    if not np.isfinite(vals[i]):
        raise ValueError("no k in range overlaps enough points")
    a, b = np.log(grid[max(i - 1, 0)]), np.log(grid[min(i + 1, len(grid) - 1)])
    g = (np.sqrt(5.0) - 1.0) / 2.0
    c, d = b - g * (b - a), a + g * (b - a)
    for _ in range(60):
        if f(np.exp(c)) < f(np.exp(d)):
            b = d
        else:
            a = c
        c, d = b - g * (b - a), a + g * (b - a)
    k = float(np.exp(0.5 * (a + b)))
    m, n = rescaled_mismatch(t_ref, e_ref, t, e, k)
    return k, m, n


def c4_integrals(c4, n_max=3, err=None, k_sigma=3.0):
    """I_n = integral over r of r^n C4(r) (Sec. 3), n = 0..n_max, for C4 given
    at the lattice distances r = 0..L-1 of a periodic lattice (C4(r) = C4(L - r)).
    The integral is taken as the sum over r = 0..L/2, stopped before the first
    r at which C4 is no longer above its noise: not positive, or, when the
    standard errors err[r] of C4 are given, not above k_sigma of them (the paper
    leaves the estimation details to its references). Returns (I_0..I_n_max,
    the last r summed)."""
    c4 = np.asarray(c4, np.float64)
    floor = np.zeros_like(c4) if err is None else k_sigma * np.asarray(err, np.float64)
    r_max = len(c4) // 2
    stop = r_max
    for r in range(1, r_max + 1):
        if c4[r] <= floor[r]:
            stop = r - 1
            break
    r = np.arange(stop + 1, dtype=np.float64)
    return np.array([np.sum(r ** n * c4[:stop + 1]) for n in range(n_max + 1)]), stop


def xi(c4, n=1, err=None, k_sigma=3.0):
    """Characteristic length xi_{n,n+1} = I_{n+1} / I_n (Eq. (xi-def)); n = 1
    gives the coherence length xi_12."""
    I, _ = c4_integrals(c4, n + 1, err, k_sigma)
    return float(I[n + 1] / I[n])


def xi_of_samples(c4_samples, n=1, k_sigma=3.0):
    """xi_{n,n+1} of the sample average of C4 (rows: samples), the integrals cut
    where the average falls below k_sigma standard errors of the mean."""
    c = np.asarray(c4_samples, np.float64)
    err = c.std(axis=0, ddof=1) / np.sqrt(c.shape[0]) if c.shape[0] > 1 else None
    return xi(c.mean(axis=0), n, err, k_sigma)
