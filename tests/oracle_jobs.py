"""Oracle runs of single pool jobs, importable by spawned worker processes.

A served or batched job is what micsa_create(L, 1, R, seed) followed by one
run over its schedule computes; the pool measures it after every tick of K
sweeps of the job's own clock and after its last sweep, and keeps the lowest
energy per replica (ties: the earliest) with its configuration.
"""
import numpy as np

import oracle


def job_with_best(args):
    """(L, R, seed, schedule, interval, K) -> final H_EA, H_aux, spins [R, N],
    daemons [R, N], lowest H_EA, its sweep count and configuration [R, N]."""
    L, R, seed, sched, interval, K = args
    orc = oracle.Oracle()
    st = orc.create(L, 1, R, seed)
    n = len(sched)
    best = np.full(R, 1 << 62, np.int64)
    best_t = np.zeros(R, np.int64)
    best_s = np.zeros((R, L ** 3), np.int8)
    e = a = None
    for k0 in range(0, n, K):
        orc.run(st, sched[k0:k0 + K], interval)
        e, a, _ = orc.measure(st)
        for rr in range(R):
            if e[rr] < best[rr]:
                best[rr], best_t[rr] = e[rr], st["t"]
                best_s[rr] = st["s"][0, rr]
    return e, a, st["s"][0].copy(), st["m"][0].copy(), best, best_t, best_s
