"""Write the stored expected values of the full-size parity tests.

Calls only the CPU oracle (``oracle/``): nothing here comes from the CUDA path.
Each output file names the workload it holds; the workloads are the synthetic
stand-ins for the paper's runs (Sec. 3: a quench to T = 0.7 from a fully
disordered start, daemons refreshed every 10 sweeps):

  quench_L32_64x2.txt    L = 32, 64 samples x 2 replicas, seed 2, T = 0.7, 10^4
                         sweeps: H_EA and Q_ab at t = 0 and floor(10^(k/8)),
                         k = 0..32; final H_aux and SHA-256 of the final spins
                         and daemons
  quench_L160_1x2.txt    L = 160, 1 sample x 2 replicas, seed 3, T = 0.7, the
                         first 10^3 sweeps: H_EA, H_aux, Q every 100 sweeps and
                         SHA-256 of spins and daemons at t = 100, 500, 1000
  batched_subset16.txt   the first 16 of the 256 batched lattices (numpy
                         default_rng(4): L from {16, 24, 32, 48, 64}, refresh
                         interval 5..20, a seed each), 2 replicas, linear
                         anneal 2.5 -> 0.5 over 2 x 10^4 sweeps: final H_EA,
                         H_aux and SHA-256 of the final spins and daemons

State hashes are over the natural layout (site = (z L + y) L + x) of int8
spins [S][R][N] and uint8 daemons m [S][R][N]; equal hashes mean equal bytes.

    python tests/golden/make_golden.py [quench_l32] [quench_l160] [batched]
"""
import hashlib
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def log_grid(t_max=10_000):
    """t = 0 and floor(10^(k/8)) for k = 0..32 (eight points per decade)."""
    return sorted({0} | {int(10 ** (k / 8)) for k in range(33)} | {t_max})


def linear_anneal(T0, T1, n):
    """Reading 4: T(k) = T0 + (T1 - T0) * (k / (n - 1)) in IEEE double."""
    if n <= 1:
        return np.full(n, float(T0))
    k = np.arange(n, dtype=np.float64)
    return float(T0) + (float(T1) - float(T0)) * (k / float(n - 1))


def batched_instances(n=256):
    rng = np.random.default_rng(4)
    Ls = rng.choice([16, 24, 32, 48, 64], n)
    rs = rng.integers(5, 21, n)
    seeds = rng.integers(1, 2 ** 62, n)
    return [(int(L), int(r), int(s)) for L, r, s in zip(Ls, rs, seeds)]


def quench_l32():
    import oracle
    O = oracle.Oracle()
    L, S, R, T, r = 32, 64, 2, 0.7, 10
    st = O.create(L, S, R, 2)
    lines = ["# L=32 quench: 64 samples x 2 replicas, seed 2, T=0.7, refresh every 10, 1e4 sweeps",
             "# written by tests/golden/make_golden.py (the CPU oracle only)",
             "# t <H_EA per (sample, replica), sample-major> | <Q_ab per sample>"]
    t_prev = 0
    for t in log_grid():
        if t > t_prev:
            O.run(st, np.full(t - t_prev, T), r)
            t_prev = t
        e, a, q = O.measure(st)
        lines.append(f"t {t} E {' '.join(map(str, e))} Q {' '.join(map(str, q))}")
    e, a, q = O.measure(st)
    lines.append(f"final_aux {' '.join(map(str, a))}")
    lines.append(f"final_spins_sha256 {sha(st['s'])}")
    lines.append(f"final_daemons_sha256 {sha(st['m'])}")
    return "quench_L32_64x2.txt", lines


def quench_l160():
    import oracle
    O = oracle.Oracle()
    L, S, R, T, r = 160, 1, 2, 0.7, 10
    st = O.create(L, S, R, 3)
    lines = ["# L=160 quench: 1 sample x 2 replicas, seed 3, T=0.7, refresh every 10, first 1000 sweeps",
             "# written by tests/golden/make_golden.py (the CPU oracle only)",
             "# t E <H_EA per replica> A <H_aux per replica> Q <Q_01> [S <sha256 spins> M <sha256 daemons>]"]
    for t in range(100, 1001, 100):
        O.run(st, np.full(100, T), r)
        e, a, q = O.measure(st)
        line = f"t {t} E {' '.join(map(str, e))} A {' '.join(map(str, a))} Q {' '.join(map(str, q))}"
        if t in (100, 500, 1000):
            line += f" S {sha(st['s'])} M {sha(st['m'])}"
        lines.append(line)
    return "quench_L160_1x2.txt", lines


def _batched_job(args):
    idx, L, r, seed, n = args
    import oracle
    O = oracle.Oracle()
    st = O.create(L, 1, 2, seed)
    O.run(st, linear_anneal(2.5, 0.5, n), r)
    e, a, _ = O.measure(st)
    return (f"job {idx} L {L} r {r} seed {seed} E {' '.join(map(str, e))} A {' '.join(map(str, a))} "
            f"S {sha(st['s'])} M {sha(st['m'])}")


def batched(n_jobs=16, n_sweeps=20_000, procs=None):
    inst = batched_instances()[:n_jobs]
    jobs = [(i, L, r, s, n_sweeps) for i, (L, r, s) in enumerate(inst)]
    jobs.sort(key=lambda j: -j[1])  # the largest lattices first
    with mp.get_context("spawn").Pool(procs or os.cpu_count()) as pool:
        rows = pool.map(_batched_job, jobs, chunksize=1)
    rows.sort(key=lambda line: int(line.split()[1]))
    lines = ["# batched subset: the first 16 of the 256 lattices of default_rng(4) (L, refresh interval, seed),",
             "# 2 replicas, linear anneal 2.5 -> 0.5 over 2e4 sweeps; final state",
             "# written by tests/golden/make_golden.py (the CPU oracle only)"] + rows
    return "batched_subset16.txt", lines


def write(name, lines):
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", name, flush=True)


if __name__ == "__main__":
    which = sys.argv[1:] or ["quench_l160", "batched", "quench_l32"]
    for w in which:
        write(*{"quench_l32": quench_l32, "quench_l160": quench_l160, "batched": batched}[w]())
