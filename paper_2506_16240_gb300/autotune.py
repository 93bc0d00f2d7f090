"""Autotuner for the launch shape of the sweep kernels.

For a lattice shape (L, samples, replicas) it times the candidate launch
shapes (32-bit words per thread, threads per block, grid-stride cap) and, for
lattices that fit in shared memory, the resident engines, and for L a multiple
of 32 the bit-plane engine (words per thread, replicas per thread), on a short run of
sweeps of that very shape, and keeps the fastest. Every choice computes the
same bits, so tuning never changes results. Choices are cached in a JSON file
keyed by device name and shape (``MICSA_AUTOTUNE_CACHE``, default
``~/.cache/micsa_autotune.json``).
"""
import itertools
import json
import os

import numpy as np

from . import Micsa, MicsaError

CACHE = os.environ.get("MICSA_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "micsa_autotune.json"))


def _key(device_name, L, S, R):
    return f"{device_name}|L={L}|S={S}|R={R}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = f"{CACHE}.{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass  # a read-only home only loses the cache


def candidates(L, R=1):
    out = [{"engine": "stream", "words_per_thread": nw, "block": blk, "blocks_per_sm": bps}
           for nw, blk, bps in itertools.product([4, 2], [64, 128, 256], [-1, 0, 2, 3, 4, 5])]
    # register-capped variant (64 registers, up to 8 blocks of 128 per SM)
    out += [{"engine": "stream", "words_per_thread": nw | 256, "block": blk, "blocks_per_sm": bps}
            for nw, blk, bps in itertools.product([4, 2], [64, 128], [-1, 0, 4, 6, 8])]
    if R >= 2:  # replica groups as concurrent kernel chains in the graphs
        out += [{"engine": "stream", "words_per_thread": 4, "block": blk, "blocks_per_sm": bps, "chains": 2}
                for blk, bps in itertools.product([64, 128, 256], [-1, 0, 3, 4])]
        # the block sizes between: other wave and tail shapes of the one-chunk-per-thread grid
        out += [{"engine": "stream", "words_per_thread": 4, "block": blk, "blocks_per_sm": 0, "chains": 2}
                for blk in (96, 160, 192, 224)]
        out += [{"engine": "stream", "words_per_thread": 4, "block": blk, "blocks_per_sm": bps, "chains": 2,
                 "graph_sweeps": 256} for blk, bps in itertools.product((64, 128), (-1, 0))]
        # two rows per thread (rows without padding)
        out += [{"engine": "stream", "words_per_thread": nw | 512, "block": blk, "blocks_per_sm": -1, "chains": 2}
                for nw, blk in itertools.product([2, 4], [64, 128])]
        # every replica of a chunk in one thread (rows without padding)
        out += [{"engine": "stream", "words_per_thread": nw | 1024, "block": blk, "blocks_per_sm": bps}
                for nw, blk, bps in itertools.product([2, 4], [64, 128, 256], [-1, 0])]
    out += [{"engine": "onchip", "words_per_thread": nw} for nw in (4, 1)]  # where the state fits on chip
    out += [{"engine": "tma", "chains": c} for c in (1, 2) if c <= R]  # where the row pitch allows TMA tiles
    if L <= 40:
        out.append({"engine": "resident"})
    if L <= 32:
        out.append({"engine": "multispin"})
    if L % 32 == 0:
        rpts = sorted({0} | {r for r in (1, 2, 4, 8, 16, 32) if r <= R})
        out += [{"engine": "multispin_global", "words_per_thread": nw, "replicas_per_thread": rpt}
                for nw, rpt in itertools.product([1, 2, 4, 2 | 256, 4 | 256], rpts)]
        if R >= 2:
            out += [{"engine": "multispin_global", "words_per_thread": nw, "replicas_per_thread": 0, "chains": 2}
                    for nw in (1, 2, 4)]
    return out


def apply(g, choice, resident_sweeps=256):
    g.set_replica_chains(choice.get("chains", 1))
    if choice["engine"] == "stream":
        g.set_engine("stream")
        g.set_launch_config(choice["words_per_thread"], choice["block"], choice["blocks_per_sm"], True,
                            choice.get("graph_sweeps", 64))
    elif choice["engine"] == "tma":
        g.set_engine("tma")
    elif choice["engine"] == "onchip":
        g.set_launch_config(choice["words_per_thread"], 128, -1, True, 64)
        g.set_engine("onchip", 2048)
    elif choice["engine"] == "multispin_global":
        g.set_engine("multispin_global")
        g.set_launch_config(choice["words_per_thread"], 128, -1, True, 64)
        g.set_multispin_replicas(choice["replicas_per_thread"])
    else:
        g.set_engine(choice["engine"], resident_sweeps)


def tune(g, torch, stream, sweeps=400, T=0.7, refresh_interval=10, use_cache=True, engines=None):
    """Pick and apply the fastest launch shape for handle g; returns the choice
    with its measured spin-flips/ns. The handle's state is advanced (t moves).
    engines: the engine names to consider (None: all)."""
    name = torch.cuda.get_device_name()
    key = _key(name, g.L, g.S, g.R) + ("" if engines is None else "|" + ",".join(sorted(engines)))
    cache = _load() if use_cache else {}
    if key in cache:
        apply(g, cache[key])
        return dict(cache[key], cached=True)
    sched = np.full(sweeps, T)
    best = None
    for c in candidates(g.L, g.R):
        if engines is not None and c["engine"] not in engines:
            continue
        try:
            apply(g, c)
            # warm-up as long as the timed run: the sweep table is sized and the
            # graph of this shape captured before timing (one-time setup costs)
            g.run(sched, refresh_interval)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.run(sched, refresh_interval)
            e1.record(stream)
            torch.cuda.synchronize()
        except MicsaError:  # the lattice does not fit this engine, or its launch was refused
            continue
        rate = g.L ** 3 * g.S * g.R * sweeps / (e0.elapsed_time(e1) * 1e6)
        if best is None or rate > best[1]:
            best = (c, rate)
    choice = dict(best[0], flips_per_ns=best[1])
    apply(g, choice)
    if use_cache:
        cache[key] = choice
        _store(cache)
    return dict(choice, cached=False)


# ----------------------------------------------------------------- pool --
def pool_candidates():
    """(max_words, chains) shapes of the pool's streaming half-sweeps."""
    return [{"max_words": w, "chains": c, "blocks_per_sm": 0} for w, c in itertools.product([4, 2, 1], [1, 2, 3, 4])]


def apply_pool(pool, choice):
    """Apply a pool choice (the shared-memory bit-plane setting applies to the
    jobs admitted afterwards: apply it before submitting)."""
    pool.set_shape(choice["max_words"], choice["chains"])
    pool.set_launch_config(choice.get("blocks_per_sm", 0))  # 0: as many blocks as fit
    if "smem_planes" in choice:
        budget, bps = choice["smem_planes"][:2]
        pool.set_smem_planes(min(budget, pool.smem_planes()[1]), bps)
        if len(choice["smem_planes"]) > 2:
            pool.set_smem_clusters(bool(choice["smem_planes"][2]))


def smem_plane_candidates(max_budget):
    """(budget bytes, CTAs per SM, units over clusters) of the shared-memory bit-plane
    path: off; the whole budget (a unit takes as many replicas of a job as fit), in
    one CTA or split over a cluster of one CTA per z word; 100 KB (units of one
    replica up to L = 64: more, shorter units, so the tick is not held up by the
    longest one), in one CTA or over a cluster; 60 KB in one CTA (one replica of
    L <= 48, the L = 56 and 64 jobs on the global bit planes). CTAs of 512 threads,
    one per SM."""
    half = min(max_budget, 100 << 10)
    return [(0, 1, False), (max_budget, 1, False), (max_budget, 1, True), (half, 1, False), (half, 1, True),
            (min(max_budget, 60 << 10), 1, False)]


def time_pool_ticks(pool, ticks, clock):
    """Seconds for `ticks` ticks of the pool after one untimed tick (which
    uploads the tables and captures the tick's graph for the current shape)."""
    pool.tick()
    pool.wait()
    t0 = clock()
    for _ in range(ticks):
        pool.tick()
    pool.wait()
    return clock() - t0


def tune_pool(pool, ticks=2, blocks=(3, 4, 5, 6, 8), clock=None):
    """Pick and apply the fastest pool shape for the jobs admitted to `pool`:
    first (words per thread cap, chains) at the default grid, then blocks per SM
    at the best shape. Every choice computes the same bits, so the jobs just
    advance while they are timed; none of them should finish during the tuning
    (give them more sweeps than (1 + ticks) x tick_sweeps x the candidates).
    Returns the choice with its time per tick."""
    import time
    clock = clock or time.perf_counter
    best = None
    for c in pool_candidates():
        apply_pool(pool, c)
        dt = time_pool_ticks(pool, ticks, clock) / ticks
        if best is None or dt < best[0]:
            best = (dt, dict(c))
    shape = best[1]
    for bps in blocks:
        c = dict(shape, blocks_per_sm=bps)
        apply_pool(pool, c)
        dt = time_pool_ticks(pool, ticks, clock) / ticks
        if dt < best[0]:
            best = (dt, c)
    apply_pool(pool, best[1])
    return dict(best[1], s_per_tick=best[0])


def tune_pool_for_jobs(pool_factory, jobs, ticks=2, clock=None, smem=None):
    """Tune on scratch pools: pool_factory() makes one, `jobs` are submit()
    argument tuples (L, R, seed, n_sweeps, interval, T_start, T_end) whose sweep
    counts are raised so that no job finishes while the candidates run. For each
    shared-memory bit-plane setting (smem: list of (budget, CTAs per SM); None:
    smem_plane_candidates) the jobs are admitted to a fresh scratch pool and its
    shape tuned (tune_pool). Returns the fastest choice (apply it to the real pool
    with apply_pool before submitting)."""
    n_cand = len(pool_candidates()) + 5
    best = None
    settings = smem
    for k in range(len(settings) if settings is not None else len(smem_plane_candidates(1 << 20))):
        with pool_factory() as p:
            if settings is None:
                settings = smem_plane_candidates(p.smem_planes()[1])
            budget, bps = settings[k][:2]
            p.set_smem_planes(budget, bps)
            if len(settings[k]) > 2:
                p.set_smem_clusters(bool(settings[k][2]))
            K = p.tick_sweeps
            long = (1 + ticks) * K * (n_cand + 2)  # candidates x (warm-up + timed ticks), with a margin
            for L, R, seed, _, interval, T0, T1 in jobs:
                if p.submit(L, R, seed, long, interval, T0, T1) is None:
                    break  # the scratch pool is full: tune on what fits
            c = dict(tune_pool(p, ticks=ticks, clock=clock), smem_planes=list(settings[k]))
        if best is None or c["s_per_tick"] < best["s_per_tick"]:
            best = c
    return best
