"""GPU tests of the batched pool and the serving loop.

A pool job must compute exactly what a single handle computes for the same
(L, R, seed, schedule, refresh interval), whatever slot it gets and whatever
runs beside it; its best configuration must be the oracle's lowest-energy
state at the tick boundaries. Admission must respect the arena size.
"""
import numpy as np
import pytest

import oracle
import oracle_jobs
import paper_2506_16240_gb300 as micsa
from paper_2506_16240_gb300 import serve

pytestmark = pytest.mark.gpu

O = oracle.Oracle()


def assert_final_state(res, st, what):
    """Final spins and daemons of a pool job equal the oracle's, element by element."""
    np.testing.assert_array_equal(res["spins"], st["s"][0], err_msg=f"spins {what}")
    np.testing.assert_array_equal(res["daemons"], st["m"][0], err_msg=f"daemons {what}")


def single_handle(L, R, seed, n, interval, T0, T1):
    sched = micsa.linear_schedule(T0, T1, n)
    with micsa.Micsa(L, 1, R, seed) as g:
        g.run(sched, interval)
        e, a, _ = g.measure()
        s, _, _ = g.get_state()
    return e, a, s


def run_pool(jobs, K=16, arena=1 << 28, max_jobs=64, order=None, shape=None, reshape=None, planes=None, smem=None):
    """Run jobs to completion; shape: (max_words, chains, blocks_per_sm) set
    before the submissions, reshape: one set after the first tick; planes: the
    bit-plane path on or off for the jobs (None: the pool's default, on); smem:
    (budget bytes, blocks per SM) of the shared-memory bit-plane kernel (None:
    the default, the device's largest budget)."""
    with micsa.Pool(arena, max_jobs, K) as p:
        if planes is not None:
            p.set_planes(planes)
        if smem is not None:
            p.set_smem_planes(*smem[:2])
            if len(smem) > 2:
                p.set_smem_clusters(smem[2])
        if shape:
            p.set_shape(shape[0], shape[1])
            p.set_launch_config(shape[2])
        ids = {}
        for idx in (order or range(len(jobs))):
            jid = p.submit(*jobs[idx])
            assert jid is not None
            ids[idx] = jid
        results = {}
        ticks = 0
        while len(results) < len(jobs):
            p.tick()
            ticks += 1
            if reshape and ticks == 1:
                p.set_shape(reshape[0], reshape[1])
                p.set_launch_config(reshape[2])
            for idx, jid in ids.items():
                if idx not in results:
                    r = p.poll(jid, final_state=True)
                    if r is not None:
                        results[idx] = r
        return results


JOBS = [  # (L, R, seed, n_sweeps, interval, T_start, T_end)
    (8, 1, 11, 100, 10, 3.0, 0.5), (16, 2, 12, 77, 5, 2.5, 0.5), (10, 3, 13, 40, 7, 2.0, 1.0),
    (32, 2, 14, 50, 20, 2.5, 0.5), (6, 4, 15, 33, 1, 3.0, 0.3), (18, 1, 16, 64, 9, 2.5, 0.4),
    (24, 2, 17, 16, 16, 1.5, 1.5), (30, 1, 18, 5, 3, 2.0, 0.7),
    (34, 2, 19, 30, 6, 2.0, 0.6), (40, 1, 20, 21, 4, 2.0, 1.0),  # too big for the resident kernel
]


def test_pool_jobs_equal_single_handle_runs():
    res = run_pool(JOBS)
    for idx, (L, R, seed, n, interval, T0, T1) in enumerate(JOBS):
        e, a, _ = single_handle(L, R, seed, n, interval, T0, T1)
        np.testing.assert_array_equal(res[idx]["energy"], e, err_msg=str(JOBS[idx]))
        np.testing.assert_array_equal(res[idx]["aux"], a, err_msg=str(JOBS[idx]))
        assert res[idx]["sweeps_done"] == n


def test_pool_result_independent_of_slot_and_neighbours():
    alone = run_pool([JOBS[1]])[0]
    mixed = run_pool(JOBS, order=list(reversed(range(len(JOBS)))))[1]
    for k in ("energy", "aux", "best_energy", "best_t"):
        np.testing.assert_array_equal(alone[k], mixed[k], err_msg=k)
    np.testing.assert_array_equal(alone["best_spins"], mixed["best_spins"])


# streamed by the pool half-sweep kernel (too big for the shared-memory kernel):
# one job per (words per thread, rows with or without padding) variant
JOBS_STREAMED = [  # (L, R, seed, n_sweeps, interval, T_start, T_end)
    (42, 1, 21, 12, 5, 2.0, 0.8),   # 2 words per thread, padded rows
    (48, 2, 22, 13, 4, 2.5, 0.5),   # 2 words, rows without padding
    (50, 1, 23, 9, 3, 2.0, 1.0),    # 1 word, padded rows
    (56, 1, 26, 7, 2, 1.5, 1.5),    # 1 word, rows without padding
    (58, 1, 24, 11, 10, 2.0, 0.6),  # 4 words, padded rows
    (64, 2, 25, 12, 6, 2.5, 0.5),   # 4 words, rows without padding
]


def test_pool_streamed_variants_match_oracle():
    res = run_pool(JOBS_STREAMED, K=5, planes=False)  # the byte kernel for every job
    for idx, (L, R, seed, n, interval, T0, T1) in enumerate(JOBS_STREAMED):
        st = O.create(L, 1, R, seed)
        O.run(st, micsa.linear_schedule(T0, T1, n), interval)
        e, a, _ = O.measure(st)
        np.testing.assert_array_equal(res[idx]["energy"], e, err_msg=str(JOBS_STREAMED[idx]))
        np.testing.assert_array_equal(res[idx]["aux"], a, err_msg=str(JOBS_STREAMED[idx]))
        assert_final_state(res[idx], st, JOBS_STREAMED[idx])
        assert res[idx]["sweeps_done"] == n


def test_batched_workload_in_one_pool_sampled_jobs_match_oracle():
    """The batched workload's 256 lattices (L drawn from {16, 24, 32, 48, 64}, 2
    replicas, refresh interval 5..20, a seed each, from the same generator) in one
    pool with ticks of 256 sweeps, on a short anneal 2.5 -> 0.5 of 40 sweeps: for
    one job of each L the final energies equal the oracle's."""
    rng = np.random.default_rng(4)
    Ls = rng.choice([16, 24, 32, 48, 64], 256)
    rs = rng.integers(5, 21, 256)
    seeds = rng.integers(1, 2 ** 62, 256)
    n = 40
    with micsa.Pool(8 << 30, 512, 256) as p:
        ids = [p.submit(int(L), 2, int(s), n, int(r), 2.5, 0.5) for L, r, s in zip(Ls, rs, seeds)]
        assert all(i is not None for i in ids)
        res = {}
        while len(res) < len(ids):
            p.tick()
            for i, jid in enumerate(ids):
                if i not in res:
                    r = p.poll(jid, best_spins=False, final_state=True)
                    if r is not None:
                        res[i] = r
    for L in (16, 24, 32, 48, 64):
        i = int(np.flatnonzero(Ls == L)[0])
        st = O.create(L, 1, 2, int(seeds[i]))
        O.run(st, micsa.linear_schedule(2.5, 0.5, n), int(rs[i]))
        e, a, _ = O.measure(st)
        np.testing.assert_array_equal(res[i]["energy"], e, err_msg=f"L={L}")
        np.testing.assert_array_equal(res[i]["aux"], a, err_msg=f"L={L}")
        assert_final_state(res[i], st, f"L={L}")


@pytest.mark.parametrize("job", [JOBS[0], JOBS[2], JOBS[5], JOBS[8], JOBS_STREAMED[1], JOBS_STREAMED[4],
                                 JOBS_STREAMED[5], (64, 2, 35, 40, 6, 2.5, 0.5)])
def test_pool_best_configuration_matches_oracle(job):
    L, R, seed, n, interval, T0, T1 = job
    K = 16
    r = run_pool([job], K=K)[0]
    st = O.create(L, 1, R, seed)
    sched = micsa.linear_schedule(T0, T1, n)
    best = np.full(R, 1 << 62, np.int64)
    best_t = np.zeros(R, np.int64)
    best_s = np.zeros((R, L ** 3), np.int8)
    for k0 in range(0, n, K):
        O.run(st, sched[k0:k0 + K], interval)
        e, a, _ = O.measure(st)
        for rr in range(R):
            if e[rr] < best[rr]:
                best[rr], best_t[rr] = e[rr], st["t"]
                best_s[rr] = st["s"][0, rr]
    np.testing.assert_array_equal(r["best_energy"], best)
    np.testing.assert_array_equal(r["best_t"], best_t)
    np.testing.assert_array_equal(r["best_spins"], best_s)
    np.testing.assert_array_equal(r["energy"], e)
    np.testing.assert_array_equal(r["aux"], a)
    assert_final_state(r, st, job)


def test_admission_is_limited_by_arena_memory():
    job = (64, 2, 21, 40, 10, 2.0, 0.5)
    need = micsa.Pool.job_bytes(64, 2, 40, 10)
    assert 2.5 * need > (1 << 20)
    with micsa.Pool(arena_bytes=int(2.5 * need), max_jobs=8, tick_sweeps=16) as p:
        a = p.submit(*job)
        b = p.submit(*job[:2], 22, *job[3:])
        assert a is not None and b is not None
        assert p.submit(*job[:2], 23, *job[3:]) is None  # no room for a third
        free_before = p.stats()["free_bytes"]
        while p.poll(a) is None:
            p.tick()
        assert p.stats()["free_bytes"] > free_before
        c = p.submit(*job[:2], 23, *job[3:])
        assert c is not None
        for jid in (b, c):
            while p.poll(jid) is None:
                p.tick()
        assert p.stats()["live_jobs"] == 0


def test_finished_lists_exactly_the_completed_jobs():
    with micsa.Pool(1 << 26, 8, 16) as p:
        short = p.submit(8, 1, 1, 16, 4, 2.0, 1.0)   # one tick
        long_ = p.submit(34, 1, 2, 64, 4, 2.0, 1.0)  # four ticks (streaming part)
        p.tick()
        p.wait()
        assert p.finished() == [short]
        assert p.poll(short) is not None and p.poll(long_) is None
        for _ in range(3):
            p.tick()
        p.wait()
        assert p.finished() == [long_]
        assert p.poll(long_)["sweeps_done"] == 64


def test_pool_rejects_bad_jobs():
    with micsa.Pool(1 << 24, 4, 8) as p:
        with pytest.raises(micsa.MicsaError):
            p.submit(7, 1, 1, 10, 10, 1.0, 1.0)  # odd L
        with pytest.raises(micsa.MicsaError):
            p.submit(8, 9, 1, 10, 10, 1.0, 1.0)  # too many replicas
        with pytest.raises(micsa.MicsaError):
            p.submit(8, 1, 1, 10, 0, 1.0, 1.0)  # interval 0


def test_serving_stream_results_match_alone():
    """Requests arriving while others run are admitted into the running batch;
    each result equals the job run alone."""
    reqs = serve.poisson_stream(24, rate_hz=400.0, seed=5, L_range=(8, 24), sweeps_range=(20, 300),
                                replicas_range=(1, 3))
    with micsa.Pool(1 << 26, 6, 16) as p:  # 6 slots: later requests queue and join mid-stream
        done = serve.Server(p).serve(reqs, realtime=True)
    assert len(done) == len(reqs)
    overlapped = sum(1 for r in done if any(o.admitted < r.admitted < o.done for o in done if o is not r))
    assert overlapped > 0
    for r in done:
        e, a, _ = single_handle(r.L, r.n_replicas, r.seed, r.n_sweeps, r.refresh_interval, r.T_start, r.T_end)
        np.testing.assert_array_equal(r.result["energy"], e)
        np.testing.assert_array_equal(r.result["aux"], a)
    s = serve.summarize(done, 1.0)
    assert s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_served_stream_up_to_l96_r4_matches_oracle():
    """The serving configuration's size range (even L up to 96, 1..4 replicas,
    anneal 3.0 -> 0.3, refresh every 10) on short jobs: requests arrive while
    others run and join the running batch; every result -- final energies,
    daemon energies, final spins and daemons, the lowest energy, its time and
    configuration -- equals the oracle's, element by element."""
    import multiprocessing as mp
    K = 16
    reqs = serve.poisson_stream(14, rate_hz=300.0, seed=55, L_range=(16, 96), sweeps_range=(24, 90),
                                replicas_range=(1, 4))
    reqs[0].L, reqs[0].n_replicas = 96, 4  # the corner of the range, always present
    reqs[1].L, reqs[1].n_replicas = 94, 3  # a ragged bit-plane-ineligible large job
    with micsa.Pool(1 << 30, 5, K) as p:  # 5 slots: later requests queue and join mid-stream
        done = serve.Server(p, keep_spins=True, final_state=True).serve(reqs, realtime=True)
    assert len(done) == len(reqs)
    overlapped = sum(1 for r in done if any(o.admitted < r.admitted < o.done for o in done if o is not r))
    assert overlapped > 0
    args = [(r.L, r.n_replicas, r.seed, micsa.linear_schedule(r.T_start, r.T_end, r.n_sweeps), r.refresh_interval, K)
            for r in done]
    with mp.get_context("spawn").Pool(min(len(args), 16)) as workers:  # spawn: this process holds a CUDA context
        ref = workers.map(oracle_jobs.job_with_best, args, chunksize=1)
    for r, (e, a, s, m, best, best_t, best_s) in zip(done, ref):
        what = f"L={r.L} R={r.n_replicas} sweeps={r.n_sweeps}"
        np.testing.assert_array_equal(r.result["energy"], e, err_msg=what)
        np.testing.assert_array_equal(r.result["aux"], a, err_msg=what)
        np.testing.assert_array_equal(r.result["spins"], s, err_msg=what)
        np.testing.assert_array_equal(r.result["daemons"], m, err_msg=what)
        np.testing.assert_array_equal(r.result["best_energy"], best, err_msg=what)
        np.testing.assert_array_equal(r.result["best_t"], best_t, err_msg=what)
        np.testing.assert_array_equal(r.result["best_spins"], best_s, err_msg=what)


@pytest.mark.parametrize("shape,reshape", [
    ((1, 1, 0), None), ((2, 3, 3), None), ((4, 4, 8), None), ((4, 2, 0), (1, 3, 2)), ((1, 4, 5), (4, 1, 0)),
])
def test_pool_results_identical_for_every_shape(shape, reshape):
    """Words per thread, chains and grid (also changed between ticks, while the
    jobs are live) do not change any job's result."""
    jobs = JOBS + JOBS_STREAMED
    ref = run_pool(jobs, K=4)
    res = run_pool(jobs, K=4, shape=shape, reshape=reshape)
    for idx in range(len(jobs)):
        for k in ("energy", "aux", "best_energy", "best_t", "sweeps_done"):
            np.testing.assert_array_equal(res[idx][k], ref[idx][k], err_msg=f"{jobs[idx]} {k}")
        np.testing.assert_array_equal(res[idx]["best_spins"], ref[idx]["best_spins"], err_msg=str(jobs[idx]))


def test_pool_shape_rejects_bad_values():
    with micsa.Pool(1 << 24, 4, 4) as p:
        for w, c in [(3, 2), (0, 2), (8, 1), (4, 0), (4, 5)]:
            with pytest.raises(micsa.MicsaError):
                p.set_shape(w, c)
        with pytest.raises(micsa.MicsaError):
            p.set_launch_config(65)


def test_pool_autotuner_choice_is_valid_and_exact():
    from paper_2506_16240_gb300 import autotune
    jobs = JOBS_STREAMED + JOBS[8:]
    choice = autotune.tune_pool_for_jobs(lambda: micsa.Pool(1 << 28, 64, 4), jobs, ticks=1)
    assert choice["max_words"] in (1, 2, 4) and 1 <= choice["chains"] <= 4
    assert 0 <= choice["blocks_per_sm"] <= 64 and choice["s_per_tick"] > 0
    ref = run_pool(jobs, K=4)
    res = run_pool(jobs, K=4, shape=(choice["max_words"], choice["chains"], choice["blocks_per_sm"]))
    for idx in range(len(jobs)):
        np.testing.assert_array_equal(res[idx]["energy"], ref[idx]["energy"], err_msg=str(jobs[idx]))


# every even L > 32 takes the pool's bit-plane path (on by default); z columns
# of L = 34..62 (except 64), 72, 88, 94 end in a partial word
JOBS_PLANES = [  # (L, R, seed, n_sweeps, interval, T_start, T_end)
    (64, 2, 31, 23, 5, 2.5, 0.5), (96, 1, 32, 9, 3, 2.0, 1.0), (64, 3, 33, 17, 7, 3.0, 0.3), (128, 1, 34, 6, 2, 1.5, 1.5),
    (40, 2, 36, 11, 4, 2.5, 0.5), (48, 1, 37, 13, 5, 2.0, 0.8), (56, 2, 38, 9, 3, 3.0, 0.3), (72, 1, 39, 7, 2, 1.5, 1.5),
    (88, 1, 40, 5, 5, 2.0, 1.0),
    # L not a multiple of 8: plane rows padded to whole Philox blocks (P = 4 ceil(L/8) words)
    (34, 2, 41, 9, 3, 2.5, 0.5), (36, 1, 42, 7, 2, 2.0, 1.0), (38, 3, 43, 6, 4, 3.0, 0.3), (42, 2, 44, 8, 5, 2.0, 0.8),
    (46, 1, 45, 5, 1, 1.5, 1.5), (50, 2, 46, 6, 3, 2.5, 0.5), (62, 1, 47, 7, 7, 2.0, 1.0), (94, 1, 48, 4, 2, 2.0, 1.0),
]


def test_pool_plane_jobs_match_oracle():
    res = run_pool(JOBS_PLANES, K=4)
    for idx, (L, R, seed, n, interval, T0, T1) in enumerate(JOBS_PLANES):
        st = O.create(L, 1, R, seed)
        O.run(st, micsa.linear_schedule(T0, T1, n), interval)
        e, a, _ = O.measure(st)
        np.testing.assert_array_equal(res[idx]["energy"], e, err_msg=str(JOBS_PLANES[idx]))
        np.testing.assert_array_equal(res[idx]["aux"], a, err_msg=str(JOBS_PLANES[idx]))
        assert_final_state(res[idx], st, JOBS_PLANES[idx])
        assert res[idx]["sweeps_done"] == n


_PLANE_REF = {}


def _plane_oracle(idx):
    if idx not in _PLANE_REF:
        L, R, seed, n, interval, T0, T1 = JOBS_PLANES[idx]
        st = O.create(L, 1, R, seed)
        O.run(st, micsa.linear_schedule(T0, T1, n), interval)
        _PLANE_REF[idx] = (st, O.measure(st))
    return _PLANE_REF[idx]


@pytest.mark.parametrize("smem", [(0, 1), (60 << 10, 2), (120 << 10, 1), (120 << 10, 2), (60 << 10, 1, False),
                                  (120 << 10, 1, False), (232432, 1, False)])
def test_pool_smem_plane_budgets_match_oracle(smem):
    """The shared-memory bit-plane kernels at several budgets: off; 60 KB and
    120 KB with the units split over clusters of one CTA per z word (the default)
    and in one CTA each (one replica per unit, bonds from the arena, the larger
    jobs on the global bit planes at 60 KB; one replica beside its bond planes for
    L = 40, two replicas without them for L = 48 at 120 KB), one or two CTAs per
    SM; the whole budget in one CTA; the default (whole budget, clusters) is
    covered by every other pool test. Final state, energies and daemon energies
    equal the oracle's."""
    res = run_pool(JOBS_PLANES, K=4, smem=smem)
    for idx, job in enumerate(JOBS_PLANES):
        st, (e, a, _) = _plane_oracle(idx)
        np.testing.assert_array_equal(res[idx]["energy"], e, err_msg=f"{job} {smem}")
        np.testing.assert_array_equal(res[idx]["aux"], a, err_msg=f"{job} {smem}")
        assert_final_state(res[idx], st, f"{job} {smem}")


@pytest.mark.parametrize("smem", [None, (100 << 10, 1), (100 << 10, 1, False), (232432, 1, False)])
def test_pool_smem_plane_units_split_replicas_match_oracle(smem):
    """Jobs with more replicas than one shared-memory unit holds are split into
    replica ranges (the default budget: L = 48 x 8 replicas in units of two, L = 40
    x 5 in units of two and one; 100 KB: one replica per unit); each range draws
    its own replicas' Philox streams."""
    jobs = [(48, 8, 61, 9, 4, 2.5, 0.5), (40, 5, 62, 11, 3, 3.0, 0.3), (34, 7, 63, 6, 2, 2.0, 1.0)]
    res = run_pool(jobs, K=4, smem=smem)
    for idx, (L, R, seed, n, interval, T0, T1) in enumerate(jobs):
        st = O.create(L, 1, R, seed)
        O.run(st, micsa.linear_schedule(T0, T1, n), interval)
        e, a, _ = O.measure(st)
        np.testing.assert_array_equal(res[idx]["energy"], e, err_msg=str(jobs[idx]))
        np.testing.assert_array_equal(res[idx]["aux"], a, err_msg=str(jobs[idx]))
        assert_final_state(res[idx], st, jobs[idx])


@pytest.mark.parametrize("small", [True, False])
def test_pool_small_lattices_on_both_paths_match_oracle(small):
    """Jobs with L <= 32 (odd L / 2, tiny lattices, up to eight replicas) as bit planes
    in shared memory (CTAs of 128 threads, units of several replicas) or on the
    multispin kernel: final state and energies equal the oracle's either way."""
    jobs = [(2, 3, 71, 30, 2, 3.0, 0.5), (6, 4, 72, 33, 1, 3.0, 0.3), (10, 3, 73, 40, 7, 2.0, 1.0),
            (16, 8, 74, 25, 5, 2.5, 0.5), (18, 1, 75, 64, 9, 2.5, 0.4), (24, 2, 76, 16, 16, 1.5, 1.5),
            (30, 5, 77, 21, 4, 2.0, 0.7), (32, 2, 78, 50, 20, 2.5, 0.5)]
    with micsa.Pool(1 << 28, 64, 8) as p:
        p.set_small_planes(small)
        ids = [p.submit(*j) for j in jobs]
        res = {}
        while len(res) < len(ids):
            p.tick()
            for k, jid in enumerate(ids):
                if k not in res:
                    r = p.poll(jid, final_state=True)
                    if r is not None:
                        res[k] = r
    for k, (L, R, seed, n, interval, T0, T1) in enumerate(jobs):
        st = O.create(L, 1, R, seed)
        O.run(st, micsa.linear_schedule(T0, T1, n), interval)
        e, a, _ = O.measure(st)
        np.testing.assert_array_equal(res[k]["energy"], e, err_msg=str(jobs[k]))
        np.testing.assert_array_equal(res[k]["aux"], a, err_msg=str(jobs[k]))
        assert_final_state(res[k], st, jobs[k])


def test_pool_smem_planes_rejects_bad_values():
    with micsa.Pool(1 << 24, 4, 4) as p:
        for budget, bps in [(1 << 30, 1), (1 << 16, 0), (1 << 16, 9)]:
            with pytest.raises(micsa.MicsaError):
                p.set_smem_planes(budget, bps)


@pytest.mark.parametrize("K", [3, 16])
def test_pool_results_identical_with_and_without_planes(K):
    """Resident, byte-streamed and bit-plane jobs in one pool: every result is
    the same with the bit-plane path on and off."""
    jobs = JOBS[:4] + JOBS_STREAMED + JOBS_PLANES
    on = run_pool(jobs, K=K, planes=True)
    off = run_pool(jobs, K=K, planes=False)
    for idx in range(len(jobs)):
        for k in ("energy", "aux", "best_energy", "best_t", "sweeps_done"):
            np.testing.assert_array_equal(on[idx][k], off[idx][k], err_msg=f"{jobs[idx]} {k}")
        np.testing.assert_array_equal(on[idx]["best_spins"], off[idx]["best_spins"], err_msg=str(jobs[idx]))
