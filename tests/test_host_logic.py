"""Host logic without a GPU: the continuous-batching request loop (against a
fake pool that enforces slot and memory limits), the synthetic request stream
and the autotuner's choice (against a fake handle and fake timing events)."""
import numpy as np
import pytest

from paper_2506_16240_gb300 import autotune, serve


class FakePool:
    """Slots, an arena budget of L^3 * R bytes per job, K sweeps per tick."""

    def __init__(self, max_jobs=3, arena=3 * 32 ** 3 * 2, tick_sweeps=1000):
        self.max_jobs, self.arena, self.K = max_jobs, arena, tick_sweeps
        self.tick_sweeps = tick_sweeps
        self.live, self.next_id, self.used, self.ticks = {}, 0, 0, 0
        self.admitted, self.peak_jobs, self.peak_bytes = [], 0, 0
        self.flips, self.flips_at_wait = 0, []

    def submit(self, L, R, seed, n_sweeps, interval, T0, T1):
        need = L ** 3 * R
        if len(self.live) >= self.max_jobs or self.used + need > self.arena:
            return None
        jid = self.next_id
        self.next_id += 1
        self.live[jid] = {"need": need, "left": n_sweeps, "seed": seed, "done": False, "LR": L ** 3 * R}
        self.used += need
        self.admitted.append(seed)
        self.peak_jobs = max(self.peak_jobs, len(self.live))
        self.peak_bytes = max(self.peak_bytes, self.used)
        return jid

    def tick(self):
        self.ticks += 1
        for j in self.live.values():
            self.flips += min(self.K, max(j["left"], 0)) * j["LR"]
            j["left"] -= self.K
            j["done"] = j["left"] <= 0

    def wait_ticks(self, n):
        pass

    def wait(self):
        self.flips_at_wait.append(self.flips)

    def finished(self):
        return [jid for jid, j in self.live.items() if j["done"]]

    def poll(self, jid, best_spins=False, final_state=False):
        j = self.live.pop(jid)
        self.used -= j["need"]
        return {"energy": [-j["seed"]], "seed": j["seed"]}


def _requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.choice([16, 24, 32]))
        out.append(serve.Request(arrival=0.001 * k, L=L, n_replicas=int(rng.integers(1, 3)), seed=k + 1,
                                 n_sweeps=int(rng.integers(500, 5000)), refresh_interval=10, T_start=3.0,
                                 T_end=0.3))
    return out


def test_serving_loop_admits_in_order_within_limits_and_completes_every_job():
    pool = FakePool()
    reqs = _requests(25)
    done = serve.Server(pool).serve(reqs, realtime=False)
    assert len(done) == len(reqs) and {r.seed for r in done} == {r.seed for r in reqs}
    assert pool.admitted == sorted(pool.admitted)          # FIFO admission
    assert pool.peak_jobs <= pool.max_jobs and pool.peak_bytes <= pool.arena
    assert pool.used == 0 and not pool.live                 # everything freed
    for r in done:
        assert r.result["seed"] == r.seed and r.job_id >= 0
        assert 0.0 <= r.admitted <= r.done
    s = serve.summarize(done, 1.0)
    lat = np.array([r.done - r.arrival for r in done])
    assert s["jobs"] == 25 and s["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["updates"] == sum(r.L ** 3 * r.n_replicas * r.n_sweeps for r in reqs)


def test_serving_loop_records_the_saturated_window():
    """With every request queued at once and more requests than slots, the pool is
    full until the queue empties: the window's attempts are those of the ticks run
    by then (counted by the pool itself), less than the whole stream's."""
    pool = FakePool()
    reqs = _requests(25)
    srv = serve.Server(pool)
    srv.serve(reqs, realtime=False)
    flips, secs = srv.saturated
    assert pool.flips_at_wait and flips == pool.flips_at_wait[0]
    assert 0 < flips < sum(r.updates for r in reqs) and secs > 0


def test_serving_loop_respects_arrival_times():
    pool = FakePool(max_jobs=8, arena=1 << 30)
    reqs = _requests(6)
    for k, r in enumerate(reqs):
        r.arrival = 0.02 * k
    done = serve.Server(pool).serve(reqs, realtime=True)
    assert len(done) == 6
    for r in done:
        assert r.admitted >= r.arrival - 1e-3  # never admitted before it arrived


def test_poisson_stream_follows_its_distributions():
    reqs = serve.poisson_stream(4000, rate_hz=50.0, seed=5)
    assert reqs == serve.poisson_stream(4000, rate_hz=50.0, seed=5)  # deterministic per seed
    arr = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert np.all(gaps > 0) and gaps.mean() == pytest.approx(1 / 50.0, rel=0.06)
    Ls = np.array([r.L for r in reqs])
    assert np.all(Ls % 2 == 0) and Ls.min() >= 16 and Ls.max() <= 96
    assert len(set(Ls)) == 41  # every even L in 16..96 appears
    sw = np.array([r.n_sweeps for r in reqs])
    assert sw.min() >= 999 and sw.max() <= 100_000
    assert np.mean(np.log(sw)) == pytest.approx(np.mean([np.log(1e3), np.log(1e5)]), abs=0.1)
    R = np.array([r.n_replicas for r in reqs])
    assert set(R) == {1, 2, 3, 4}
    mc = np.mean([r.updates for r in serve.poisson_stream(40000, 1.0, 9)])
    assert serve.mean_job_updates() == pytest.approx(mc, rel=0.05)


class FakeHandle:
    """Records the launch shape applied; run() charges a fake time per shape."""

    def __init__(self, L, S, R, cost):
        self.L, self.S, self.R, self.cost = L, S, R, cost
        self.engine, self.shape, self.chains, self.rpt, self.log = "stream", None, 1, 0, []

    def set_engine(self, engine, resident_sweeps=None):
        if engine == "tma" and self.L % 32:
            raise autotune.MicsaError(-1, "does not fit")
        self.engine = engine

    def set_launch_config(self, nw, block, bps, pdl, graph):
        self.shape = (nw, block, bps, graph)

    def set_replica_chains(self, c):
        self.chains = c

    def set_multispin_replicas(self, r):
        self.rpt = r

    def key(self):
        return (self.engine, self.shape, self.chains, self.rpt)

    def run(self, sched, interval):
        if self.engine == "onchip" and self.L == 160:
            raise autotune.MicsaError(-3, "launch refused")  # a candidate that fails when it runs
        self.log.append(self.key())


class FakeEvent:
    clock = []

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = len(FakeEvent.clock)
        FakeEvent.clock.append(None)

    def elapsed_time(self, other):
        return FakeEvent.costs[other.t]


class FakeTorch:
    class cuda:
        Event = FakeEvent

        @staticmethod
        def synchronize():
            pass

        @staticmethod
        def get_device_name():
            return "fake"


def test_autotuner_keeps_the_fastest_shape_and_skips_engines_that_do_not_fit(monkeypatch):
    best = ("multispin_global", (2, 128, -1, 64), 1, 4)
    h = FakeHandle(160, 1, 8, None)
    FakeEvent.clock, FakeEvent.costs = [], {}
    orig_record = FakeEvent.record

    def record(self, stream=None):  # the stop event of a timed run carries the shape's cost
        orig_record(self)
        FakeEvent.costs[self.t] = 1.0 if h.key() == best else 2.0

    monkeypatch.setattr(FakeEvent, "record", record)
    choice = autotune.tune(h, FakeTorch, None, sweeps=20, use_cache=False)
    assert (choice["engine"], choice["words_per_thread"], choice["replicas_per_thread"]) == ("multispin_global", 2, 4)
    assert h.key() == best  # the choice is applied at the end
    engines = {k[0] for k in h.log}
    assert {"stream", "multispin_global", "tma"} <= engines and "onchip" not in engines  # failed runs skipped
    h2 = FakeHandle(48, 1, 2, None)  # tma does not fit: skipped, not fatal
    FakeEvent.clock, FakeEvent.costs = [], {}
    autotune.tune(h2, FakeTorch, None, sweeps=20, use_cache=False, engines=("stream", "tma"))
    assert {k[0] for k in h2.log} == {"stream"}


def test_autotune_candidates_are_gated_by_lattice_shape():
    c160 = autotune.candidates(160, 2)
    assert not any(c["engine"] in ("resident", "multispin") for c in c160)
    assert any(c["engine"] == "multispin_global" for c in c160)
    assert any(c.get("chains") == 2 for c in c160)
    c18 = autotune.candidates(18, 1)
    assert any(c["engine"] == "resident" for c in c18) and any(c["engine"] == "multispin" for c in c18)
    assert not any(c["engine"] == "multispin_global" or c.get("chains", 1) > 1 for c in c18)


def test_time_rescaling_fit_recovers_a_planted_factor():
    """A power-law relaxation e(t) = e_inf + b t^-c sampled on a log grid, and the
    same curve with time rescaled by k = 6.034 (the paper's k* for six walkers at
    T = 0.7): the fit returns k; shifted curves or curves without overlap are
    handled."""
    from paper_2506_16240_gb300 import analysis
    t_ref = np.unique(np.round(np.logspace(0, 4, 60)))
    e_ref = -1.70 + 0.4 * t_ref ** -0.35
    for k_true in (6.034, 1.0, 2.5):
        t = np.unique(np.round(np.logspace(0, 4 - np.log10(k_true) - 0.01, 40)))
        e = -1.70 + 0.4 * (k_true * t) ** -0.35
        k, m, n = analysis.fit_time_rescaling(t_ref, e_ref, t, e)
        assert k == pytest.approx(k_true, rel=5e-3) and n >= 30 and m < 1e-6  # log-t interpolation bias
    # noise does not move the estimate much
    rng = np.random.default_rng(1)
    t = np.unique(np.round(np.logspace(0, 3, 40)))
    e = -1.70 + 0.4 * (6.0 * t) ** -0.35 + rng.normal(0, 1e-4, t.size)
    k, _, _ = analysis.fit_time_rescaling(t_ref, e_ref, t, e)
    assert k == pytest.approx(6.0, rel=0.05)
    with pytest.raises(ValueError):
        analysis.fit_time_rescaling(t_ref, e_ref, t * 1e9, e, k_range=(1.0, 2.0))


class FakeShapedPool:
    """Pool stand-in whose tick costs depend on its shape (seconds on a fake clock)."""

    def __init__(self, cost, tick_sweeps=8):
        self.cost, self.tick_sweeps = cost, tick_sweeps
        self.shape, self.blocks, self.now, self.submitted, self.ticks = (4, 2), 0, 0.0, [], 0
        self.smem = (200_000, 1, True)

    def smem_planes(self):
        return self.smem[0], 200_000, self.smem[1]

    def set_smem_planes(self, budget, bps):
        assert 0 <= budget <= 200_000 and 1 <= bps <= 8
        self.smem = (budget, bps) + self.smem[2:]

    def set_smem_clusters(self, on):
        self.smem = self.smem[:2] + (bool(on),)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def set_shape(self, w, c):
        assert w in (1, 2, 4) and 1 <= c <= 4
        self.shape = (w, c)

    def set_launch_config(self, b):
        assert 0 <= b <= 64
        self.blocks = b

    def submit(self, L, R, seed, n, interval, T0, T1):
        self.submitted.append(n)
        return len(self.submitted)

    def tick(self):
        self.ticks += 1
        self.now += self.cost(self.shape, self.blocks) * (self.smem_cost(self.smem) if hasattr(self, "smem_cost") else 1.0)

    def wait(self):
        pass


def test_pool_autotuner_picks_the_fastest_shape_then_grid():
    def cost(shape, blocks):  # fastest shape (2, 3); at that shape 5 blocks per SM beat the default
        base = 1.0 + 0.1 * abs(shape[0] - 2) + 0.05 * abs(shape[1] - 3)
        return base - (0.2 if (shape == (2, 3) and blocks == 5) else 0.0)
    fake = FakeShapedPool(cost)
    jobs = [(48, 2, 1, 100, 10, 2.5, 0.5), (64, 1, 2, 50, 5, 2.0, 1.0)]
    choice = autotune.tune_pool_for_jobs(lambda: fake, jobs, ticks=2, clock=lambda: fake.now, smem=[(0, 1)])
    assert (choice["max_words"], choice["chains"], choice["blocks_per_sm"]) == (2, 3, 5)
    assert fake.shape == (2, 3) and fake.blocks == 5  # applied
    assert choice["s_per_tick"] == pytest.approx(0.8)
    # no job may finish while the candidates run: every candidate ticks 1 + 2 times
    n_cand = len(autotune.pool_candidates()) + 5
    assert fake.ticks == 3 * n_cand
    assert all(n >= fake.ticks * fake.tick_sweeps for n in fake.submitted)


def test_pool_autotuner_picks_the_fastest_shared_memory_setting():
    """Each shared-memory bit-plane setting is set on a fresh scratch pool before
    the jobs are admitted; the fastest setting wins and is part of the choice."""
    fake = FakeShapedPool(lambda shape, blocks: 1.0)
    fake.smem_cost = lambda sm: {(0, 1, False): 1.0, (200_000, 1, False): 0.9, (200_000, 1, True): 0.8,
                                 (100 << 10, 1, False): 0.6, (100 << 10, 1, True): 0.5, (60 << 10, 1, False): 0.7}[sm]
    seen = []

    def factory():
        seen.append(len(fake.submitted))  # a fresh pool: the jobs come after the setting
        return fake
    jobs = [(48, 2, 1, 100, 10, 2.5, 0.5)]
    choice = autotune.tune_pool_for_jobs(factory, jobs, ticks=1, clock=lambda: fake.now)
    assert choice["smem_planes"] == [100 << 10, 1, True]
    assert seen == [0, 1, 2, 3, 4, 5]
    assert choice["s_per_tick"] == pytest.approx(0.5)
    applied = FakeShapedPool(lambda shape, blocks: 1.0)
    autotune.apply_pool(applied, choice)
    assert applied.smem == (100 << 10, 1, True)


def test_pool_autotuner_keeps_the_default_grid_when_no_grid_is_faster():
    fake = FakeShapedPool(lambda shape, blocks: 1.0 + (0.0 if shape == (1, 1) else 0.5) + (0.1 if blocks else 0.0))
    choice = autotune.tune_pool(fake, ticks=1, clock=lambda: fake.now)
    assert (choice["max_words"], choice["chains"], choice["blocks_per_sm"]) == (1, 1, 0)
    assert fake.shape == (1, 1) and fake.blocks == 0


def test_traffic_rows_are_well_formed():
    """Every row of the steady-state traffic table that bench.py reads has a kernel
    it knows, a digest of that kernel's sources' form, numeric byte counts and a
    capture note naming a summary that exists in profiles/; the key of a row is
    unique per kernel."""
    import os
    import re
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    seen = set()
    n = 0
    for ln in open(os.path.join(root, "profiles", "traffic.md")).read().splitlines():
        cols = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cols) < 6 or cols[0] not in bench.KERNEL_SOURCES:
            continue
        n += 1
        assert re.fullmatch(r"`[0-9a-f]{16}`", cols[2]), ln
        float(cols[3]), float(cols[4])
        summary = cols[5].split(" ")[0]
        assert os.path.isfile(os.path.join(root, "profiles", summary)), summary
        assert (cols[0], cols[1]) not in seen, ln
        seen.add((cols[0], cols[1]))
    assert n >= 2

