"""Host-side analysis of measured relaxation curves.

The paper compares MicSA with the canonical (Metropolis) dynamics by a single
time-rescaling factor k: after t_plot = k * t_MicSA the two relaxations coincide,
and k* ~ gamma for gamma walkers per spin (Sec. 3, Table (k*), Fig. 1). The
paper extracts k* from the coherence length xi_12; its integral estimators are
not given there, so here k is fitted to the energy per spin, which the paper
also compares after the rescaling (Fig. 1, Eq. (delta1)).
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
