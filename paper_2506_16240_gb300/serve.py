"""Continuous-batching serving loop over the resident pool (``micsa_pool_*``).

Requests (annealing jobs) arrive over time; each is admitted into the pool as
soon as a slot and enough arena memory are free, so that jobs arriving while
others run join the very next tick and their work overlaps on the device.
Finished jobs are polled after every tick, which returns their final and best
energies and best configurations and frees their memory for the queue.

Latency = result time - arrival time (queueing included). Throughput =
spin-flip attempts of the completed jobs / wall time of the whole stream.
"""
import time
from dataclasses import dataclass, field

import numpy as np

from . import Pool


@dataclass
class Request:
    arrival: float   # seconds after the stream starts
    L: int
    n_replicas: int
    seed: int
    n_sweeps: int
    refresh_interval: int
    T_start: float
    T_end: float
    job_id: int = -1
    admitted: float = -1.0
    done: float = -1.0
    result: dict = field(default=None, repr=False)

    @property
    def updates(self):
        return self.L ** 3 * self.n_replicas * self.n_sweeps


def poisson_stream(n_jobs, rate_hz, seed, L_range=(16, 96), sweeps_range=(1e3, 1e5),
                   replicas_range=(1, 4), T_start=3.0, T_end=0.3, refresh_interval=10):
    """Synthetic request stream: Poisson arrivals, L even-uniform, sweeps
    log-uniform, replicas uniform; every job draws its couplings from its seed."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    Ls = 2 * rng.integers(L_range[0] // 2, L_range[1] // 2 + 1, n_jobs)
    sweeps = np.exp(rng.uniform(np.log(sweeps_range[0]), np.log(sweeps_range[1]), n_jobs)).astype(np.int64)
    reps = rng.integers(replicas_range[0], replicas_range[1] + 1, n_jobs)
    seeds = rng.integers(1, 2 ** 62, n_jobs)
    return [Request(float(a), int(L), int(r), int(s), int(n), int(refresh_interval), float(T_start),
                    float(T_end))
            for a, L, r, s, n in zip(arrivals, Ls, reps, seeds, sweeps)]


def mean_job_updates(L_range=(16, 96), sweeps_range=(1e3, 1e5), replicas_range=(1, 4)):
    """Expected spin-flip attempts of one job of poisson_stream (for sizing the rate)."""
    Ls = np.arange(L_range[0], L_range[1] + 1, 2, dtype=np.float64)
    a, b = np.log(sweeps_range[0]), np.log(sweeps_range[1])
    mean_sweeps = (sweeps_range[1] - sweeps_range[0]) / (b - a)
    return float((Ls ** 3).mean() * mean_sweeps * np.mean(np.arange(replicas_range[0], replicas_range[1] + 1)))


class Server:
    def __init__(self, pool: Pool, max_pending_ticks=2, keep_spins=False, final_state=False):
        self.pool = pool
        self.max_pending = max_pending_ticks
        self.keep_spins = keep_spins
        self.final_state = final_state

    def serve(self, requests, realtime=True):
        """Run the stream to completion; returns the requests with timings and results.
        realtime=False admits every request immediately (arrival times ignored).

        Also records the saturated window: from the start until the queue first
        empties after every request has arrived, with the spin-flip attempts the
        device had completed by then (self.saturated = (updates, seconds)). With
        realtime=False and more requests than the pool holds, the pool is full for
        that whole window, so updates / seconds is its saturated capacity."""
        pending = sorted(requests, key=lambda r: r.arrival)
        queue, live, done = [], {}, []
        K = self.pool.tick_sweeps
        flips = 0  # attempts of the queued ticks (each live job advances min(K, sweeps left))
        left = {}
        self.saturated = None
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or queue or live:
            now = time.perf_counter() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                queue.append(pending[i])
                i += 1
            while queue:  # FIFO admission by free slots and free arena bytes
                r = queue[0]
                jid = self.pool.submit(r.L, r.n_replicas, r.seed, r.n_sweeps, r.refresh_interval,
                                       r.T_start, r.T_end)
                if jid is None:
                    break
                r.job_id, r.admitted = jid, time.perf_counter() - t0
                live[jid] = r
                left[jid] = r.n_sweeps
                queue.pop(0)
            if self.saturated is None and i == len(pending) and not queue:
                self.pool.wait()  # the device has run every queued tick
                self.saturated = (flips, time.perf_counter() - t0)
            if live:
                for jid, r in live.items():
                    step = min(K, left[jid])
                    left[jid] -= step
                    flips += step * r.L ** 3 * r.n_replicas
                self.pool.tick()
                self.pool.wait_ticks(self.max_pending)
                for jid in self.pool.finished():
                    res = self.pool.poll(jid, best_spins=self.keep_spins, final_state=self.final_state)
                    r = live.pop(jid)
                    r.done = time.perf_counter() - t0
                    r.result = res
                    done.append(r)
            elif i < len(pending):
                time.sleep(max(0.0, min(pending[i].arrival - now, 0.01)))
        self.wall = time.perf_counter() - t0
        return done


def summarize(done, wall):
    lat = np.array([r.done - r.arrival for r in done])
    upd = sum(r.updates for r in done)
    return {"jobs": len(done), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "wall_s": wall, "spin_flips_per_ns": upd / (wall * 1e9), "updates": int(upd)}
