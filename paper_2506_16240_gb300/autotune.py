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
        out += [{"engine": "stream", "words_per_thread": 4, "block": blk, "blocks_per_sm": -1, "chains": 2,
                 "graph_sweeps": 256} for blk in (64, 128)]
        # two rows per thread (rows without padding)
        out += [{"engine": "stream", "words_per_thread": nw | 512, "block": blk, "blocks_per_sm": -1, "chains": 2}
                for nw, blk in itertools.product([2, 4], [64, 128])]
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
