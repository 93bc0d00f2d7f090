#!/usr/bin/env python
"""Benchmark of the MicSA hot path on GB300 (one JSON line on rank 0).

Headline workload (one "step"): the single-lattice quench -- a 3D EA +-J
lattice with L = 160 (4,096,000 spins), 1 disorder sample x 2 replicas,
couplings and a random start drawn on the device from the step's seed,
quenched to T = 0.7 for 10^5 MicSA sweeps with a daemon refresh every 10
sweeps. Metric: spin-flip attempts per ns (N x replicas x samples x sweeps /
device time). The exact energy and overlap are measured after every step.

Legs on the same JSON line:
  value        device time of the step (CUDA events on the launching stream),
               state resident in HBM, L2 flushed (512 MB write) between steps
  e2e          the same job through the C ABI from pinned host buffers:
               couplings and initial spins copied in, final spins, daemons and
               observables copied out, all inside the timed region
  roofline     the plain streaming half-sweep kernel at L = 160: algorithmic
               bytes per launch over its mean duration in a timed run of
               sweeps without refresh (CUDA events, launching stream)
  dram_point   the same kernel at L = 400 (320 MB of state; each launch reads
               128 MB and writes 64 MB, so DRAM feeds it)
  metropolis   the random-number-per-update Metropolis kernel, same lattice
  quench_l32   L = 32, 64 samples x 2 replicas, T = 0.7, 10^4 sweeps, refresh
               every 10, e and q^2 measured on a log time grid (multispin
               shared-memory engine)
  batched      256 lattices, L in {16,24,32,48,64}, 2 replicas, anneal 2.5 -> 0.5
               over 2x10^4 sweeps, refresh 5..20: one pool (all jobs in each
               launch) against the per-lattice launch loop
  serving      Poisson stream of annealing jobs (L 16..96, 10^3..10^5 sweeps,
               1..4 replicas, anneal 3.0 -> 0.3) through the continuous-batching
               pool: p50/p99 latency and aggregate spin-flips/ns
  multispin_l160  the headline workload (bounded sweep count) on the bit-plane
               engine (multispin coding in HBM, 32 z per word), its launch shape
               tuned; roofline of its half-sweep kernel: algorithmic bytes
               half_sites * (7 R + 6) / 8 per launch over the mean launch time
  onchip_l160  the headline workload on the on-chip engine (the state in the
               shared memory of all SMs, halo rows exchanged through L2)
  paper_shape  L = 160, 1 sample x 128 replicas (the shape of the paper's GPU
               timings), T = 0.7, refresh every 10: bit-plane engine and the
               byte streaming engine; and one walker per spin on the log refresh
               schedule (the paper's timed configuration), bit-plane engine
  kstar        same-GPU Metropolis against MicSA with six walkers per spin on the
               same samples (L = 64, T = 0.7): the time-rescaling factor k* fitted
               to the energy relaxation
  cpu_baseline the CPU oracle on the host cores on a bounded sample of sweeps

--impl reference times the oracle itself (the deliberately slow reference).
Multi-GPU (torchrun): one independent lattice per rank (weak scaling, no
data-path collective); the barrier and the max over ranks only time the job.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "name": "L=160 EA +-J quench, 1 sample x 2 replicas, T=0.7, 1e5 sweeps, refresh every 10",
    "L": 160, "samples": 1, "replicas": 2, "T": 0.7, "sweeps": 100_000, "refresh_interval": 10,
}
METRIC = "spin-flips/ns"
L2_FLUSH_BYTES = 512 << 20


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sweeps", type=int, default=WORKLOAD["sweeps"],
                    help="sweeps per step (profiling runs only; reported numbers use the default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline leg only")
    ap.add_argument("--profile-case", choices=["stream", "chains", "chains_bps0", "chains_bps0_b96", "chains_bps0_b160",
                                               "chains_bps0_b192", "chains_bps0_b224", "chains_l400_b160",
                                               "chains_l400_bps0_b160", "single", "chains_l320",
                                               "chains_l400", "chains_l400_bps0",
                                               "multispin", "planes", "planes_r2", "planes_metro", "onchip", "tma", "pool",
                                               "batched", "plane_jobs_smem", "plane_jobs_global",
                                               "plane_jobs_smem_norefresh"],
                    help="run one small fixed workload for a profiler capture and exit")
    ap.add_argument("--pool-breakdown", action="store_true",
                    help="print tick times of the batched pool by content and shared-memory setting, and exit")
    ap.add_argument("--source-digests", action="store_true",
                    help="print the digests of the kernel sources that profiles/traffic.md rows carry")
    ap.add_argument("--serving-jobs", type=int, default=2000, help="jobs in the serving stream")
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def updates(L, S, R, sweeps):
    return L ** 3 * S * R * sweeps


def rank_seed(rank):
    """Seed of the lattice a rank runs (weak scaling: independent lattices)."""
    return 3 + 1000 * rank


def gather_ms(torch, x, rank, world, device):
    """Every rank's timing on every rank (a timing exchange only; no data-path
    collective exists: ranks run independent lattices)."""
    if world == 1:
        return [x]
    t = torch.zeros(world, dtype=torch.float64, device=device)
    t[rank] = x
    torch.distributed.all_reduce(t)
    return t.tolist()


def aggregate(world, per_rank_ms, updates_per_rank):
    """Whole-job value: all ranks' updates over the slowest rank's time."""
    total_ms = max(per_rank_ms)
    return world * updates_per_rank / (total_ms * 1e6), total_ms


# ------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


# -------------------------------------------------------- CPU oracle --
def oracle_sample(sweeps, seed=3):
    """The oracle on the headline lattice for `sweeps` sweeps: (updates, seconds)."""
    import oracle
    w = WORKLOAD
    O = oracle.Oracle()
    st = O.create(w["L"], w["samples"], w["replicas"], seed)
    t0 = time.perf_counter()
    O.run(st, np.full(sweeps, w["T"]), w["refresh_interval"])
    return updates(w["L"], w["samples"], w["replicas"], sweeps), time.perf_counter() - t0


def _oracle_worker(args):
    sweeps, seed = args
    return oracle_sample(sweeps, seed)


def cpu_baseline(target_s=12.0, parallel_s=8.0):
    """The oracle on the host cores: one process per core on independent copies
    of the headline lattice (throughput, `value`), and one process alone."""
    _, dt2 = oracle_sample(2)
    per_sweep = max(dt2 / 2, 1e-3)
    n = min(200, max(2, int(target_s / per_sweep)))
    upd, dt = oracle_sample(n)
    single = {"value": upd / (dt * 1e9), "cores": 1,
              "sample": f"{n} sweeps of the L=160 1x2 lattice, {dt:.1f} s"}
    import multiprocessing as mp
    procs = os.cpu_count() or 1
    n_each = max(2, int(parallel_s / per_sweep))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(procs) as pool:  # spawn: the parent holds a CUDA context
        res = pool.map(_oracle_worker, [(n_each, 3 + i) for i in range(procs)])
    wall = time.perf_counter() - t0
    total = sum(u for u, _ in res)
    return {"value": total / (wall * 1e9), "unit": METRIC, "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes, each {n_each} sweeps of its own L=160 1x2 lattice at T=0.7 "
                      f"(refresh every 10), single-threaded C oracle per process, {wall:.1f} s wall "
                      f"(process start included), host {os.uname().machine} with {os.cpu_count()} cores",
            "single_core": single}


def run_reference(args):
    rank, _, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOAD
    per_step = 10
    for _ in range(args.warmup):
        oracle_sample(1)
    times = [oracle_sample(per_step, seed=100 + k)[1] for k in range(args.steps)]
    value = updates(w["L"], w["samples"], w["replicas"], per_step) * args.steps / (sum(times) * 1e9)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic",
        "config": {"workload": w["name"], "L": w["L"], "samples": w["samples"], "replicas": w["replicas"],
                   "sample_per_step": f"{per_step} sweeps of the workload"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} sweeps per step of the L=160 1x2 lattice, single thread"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    return 0


# ------------------------------------------------ ncu traffic records --
# DRAM bytes of a kernel come from an ncu capture summarised in
# profiles/traffic.md, one row per (kernel, workload, launch shape), with the
# digest of the kernel's source files at capture time. A row whose digest no
# longer matches the sources describes an older kernel and is not used.
KERNEL_SOURCES = {
    "half_sweep": ["sweep_kernels.cu", "sweep_body.cuh", "micsa_device.cuh"],
    "msg_half": ["multispin.cu", "msg_body.cuh", "micsa_device.cuh"],
}


def kernel_digest(kernel):
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2506_16240_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel, key):
    """(dram bytes per half-sweep, L2 bytes per half-sweep, capture note) of the
    row `key` of profiles/traffic.md if its digest matches the current sources,
    else None."""
    try:
        lines = open(os.path.join(ROOT, "profiles", "traffic.md")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        cols = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cols) >= 6 and cols[0] == kernel and cols[1] == key:
            if cols[2].strip("`") != kernel_digest(kernel):
                return None
            return float(cols[3]), float(cols[4]), cols[5]
    return None


# --------------------------------------------------------------- GPU --
class Timer:
    def __init__(self, torch, stream):
        self.torch, self.stream = torch, stream

    def __call__(self, fn):
        t = self.torch
        e0, e1 = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        fn()
        e1.record(self.stream)
        t.cuda.synchronize()
        return e0.elapsed_time(e1)


def leg_roofline(micsa, timer, stream, L, peaks, n_plain=2048, choice=None):
    """Streaming half-sweep kernel in the launch shape `choice` (the tuned one;
    default shape if None): algorithmic bytes of one half-sweep of all
    replicas / mean time per half-sweep. With replica chains the half-sweep is
    two concurrent launches (one replica each) and the time is their span. The
    default n_plain is a multiple of the 64- and 256-sweep graphs (every timed
    half-sweep a graph node)."""
    R = 2
    g = micsa.Micsa(L, 1, R, 7, stream=stream)
    g.set_engine("stream")
    if choice is not None and choice.get("engine") == "stream":
        from paper_2506_16240_gb300 import autotune
        autotune.apply(g, choice)
        if L != WORKLOAD["L"]:
            # another lattice: the grid (grid-stride loop over the resident capacity, or
            # one thread per chunk) and block (128 or 160) that are faster at this L
            best = None
            lc0 = g.launch_config()
            for blk in (128, 160):  # the blocks whose traffic at this L is on record
                for bps in (-1, 0):
                    g.set_launch_config(lc0["words_per_thread"], blk, bps, bool(lc0["pdl"]), lc0["graph_sweeps"])
                    g.run(np.full(1, 0.7), 10)
                    # runs of whole graph replays, as in the timed region (shorter runs are
                    # direct launches, whose ranking can differ)
                    n_sel = 2 * max(64, lc0["graph_sweeps"])
                    g.run(np.full(n_sel, 0.7), 2 ** 31 - 1)
                    ms = min(timer(lambda: g.run(np.full(n_sel, 0.7), 2 ** 31 - 1)) for _ in range(2))
                    if best is None or ms < best[0]:
                        best = (ms, blk, bps)
            g.set_launch_config(lc0["words_per_thread"], best[1], best[2], bool(lc0["pdl"]), lc0["graph_sweeps"])
    g.run(np.full(1, 0.7), 10)  # t = 0 refresh; the timed sweeps below have none
    # warm-up as long as the timed run (and longer than two graph lengths), so that
    # the sweep table is sized and the sweep graph captured before the timed
    # region (one-time setup costs)
    g.run(np.full(max(600, n_plain), 0.7), 2 ** 31 - 1)
    ms = timer(lambda: g.run(np.full(n_plain, 0.7), 2 ** 31 - 1))
    shape = g.launch_config()
    g.close()
    launch_us = 1e3 * ms / (2 * n_plain)
    half_sites = L ** 3 // 2
    bytes_per_launch = half_sites * (5 * R + 1)  # per replica: s, m read + write, opposite s; bonds once
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    achieved = bytes_per_launch / (launch_us * 1e-6) / 1e9
    chains = (choice or {}).get("chains", 1)
    key = (f"L={L} R={R} chains={chains} nw={shape['words_per_thread']} block={shape['block']} "
           f"bps={shape['blocks_per_sm']}")
    rec = traffic_record("half_sweep", key)
    state_bytes = L ** 3 * (2 * R + 1)  # spins and daemons of each replica, bond bytes of the sample
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": rec[0] if rec else None, "traffic_l2": rec[1] if rec else None,
            "traffic_capture": rec[2] if rec else f"no capture of the current kernel for {key}",
            "l2_resident": state_bytes < 129e6, "state_bytes": state_bytes,
            "peak_source": "measured" if hbm else "fallback",
            "kernel": "micsa::half_sweep_kernel (streaming MicSA half-sweep, no refresh)",
            "L": L, "bytes_per_launch": bytes_per_launch, "launch_us": launch_us, "launch": shape,
            "replica_chains": chains, "flips_per_ns": updates(L, 1, R, n_plain) / (ms * 1e6)}


def plane_roofline(micsa, timer, stream, g, peaks, n_plain=1984):
    """Bit-plane half-sweep kernel of handle g (engine and shape already set):
    algorithmic bytes / mean launch time over sweeps without refresh. n_plain a
    multiple of the 64-sweep graph, so that every timed half-sweep is a graph
    node; the run's two byte <-> plane conversions stay in the timed region
    (1 of 2 n_plain / 2 launches of work each: ~0.3% at L = 160 x 128)."""
    L, S, R = g.L, g.S, g.R
    g.run(np.full(max(640, n_plain), 0.7), 2 ** 31 - 1)  # table sized, graph captured (setup costs)
    ms = timer(lambda: g.run(np.full(n_plain, 0.7), 2 ** 31 - 1))
    launch_us = 1e3 * ms / (2 * n_plain)
    half_sites = L ** 3 // 2
    # per replica: own spin, m0, m1 planes read and written, opposite spin plane read (7 bits);
    # per sample: six bond planes (6 bits)
    bytes_per_launch = half_sites * (7 * R + 6) * S // 8
    hbm = peaks.get("hbm_gbs")
    peak = hbm if hbm else 6800.0
    achieved = bytes_per_launch / (launch_us * 1e-6) / 1e9
    shape = g.launch_config()
    key = f"L={L} R={R} nw={shape['words_per_thread']}"
    rec = traffic_record("msg_half", key)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": rec[0] if rec else None, "traffic_l2": rec[1] if rec else None,
            "traffic_capture": rec[2] if rec else f"no capture of the current kernel for {key}",
            "l2_resident": L ** 3 * S * (6 * R + 12) // 16 < 129e6,  # six planes per replica, twelve of bonds
            "peak_source": "measured" if hbm else "fallback",
            "kernel": "micsa::msg_half_kernel (bit-plane MicSA half-sweep, no refresh)",
            "L": L, "replicas": R, "bytes_per_launch": bytes_per_launch, "launch_us": launch_us,
            "flips_per_ns": updates(L, S, R, n_plain) / (ms * 1e6)}


def tune_planes(g, timer, sweeps=300):
    """Fastest (words per thread, replicas per thread, replica chains) of the
    bit-plane engine."""
    best = None
    rpts = sorted({0} | {r for r in (1, 2, 4, 8, 16) if r <= g.R})
    for ch in sorted({1, min(2, g.R)}):
        for nw in (1, 2, 4):
            for rpt in rpts:
                g.set_replica_chains(ch)
                g.set_launch_config(nw, 128, -1, True, 64)
                g.set_multispin_replicas(rpt)
                g.run(np.full(20, 0.7), 10)
                ms = timer(lambda: g.run(np.full(sweeps, 0.7), 10))
                if best is None or ms < best[0]:
                    best = (ms, nw, rpt, ch)
    g.set_replica_chains(best[3])
    g.set_launch_config(best[1], 128, -1, True, 64)
    g.set_multispin_replicas(best[2])
    return {"words_per_thread": best[1], "replicas_per_thread": best[2], "chains": best[3]}


def leg_multispin_l160(micsa, timer, stream, peaks, sweeps=20_000):
    """The headline lattice and schedule on the bit-plane engine."""
    w = WORKLOAD
    L, S, R = w["L"], w["samples"], w["replicas"]
    g = micsa.Micsa(L, S, R, 5, stream=stream)
    g.set_engine("multispin_global")
    shape = tune_planes(g, timer)
    sched = np.full(sweeps, w["T"])
    g.reinit(6)
    g.run(sched, w["refresh_interval"])  # as long as the timed run: table sized, graph captured
    g.reinit(7)
    ms = timer(lambda: g.run(sched, w["refresh_interval"]))
    e, _, q = g.measure()
    roof = plane_roofline(micsa, timer, stream, g, peaks)
    g.close()
    return {"flips_per_ns": updates(L, S, R, sweeps) / (ms * 1e6), "sweeps": sweeps, "launch": shape,
            "energy_per_spin": [float(v) / L ** 3 for v in e], "roofline": roof,
            "note": "same bits as the byte engine (parity-tested); state converted to planes and back per run"}


def leg_onchip_l160(micsa, timer, stream, sweeps=5_000):
    """The headline lattice and schedule on the on-chip engine (state in the
    shared memory of all SMs, neighbour-CTA synchronisation)."""
    w = WORKLOAD
    L, S, R = w["L"], w["samples"], w["replicas"]
    g = micsa.Micsa(L, S, R, 5, stream=stream)
    best = None
    for nw in (4, 2, 1):
        g.set_launch_config(nw, 128, -1, True, 64)
        g.set_engine("onchip", 2048)
        g.run(np.full(sweeps, w["T"]), w["refresh_interval"])
        ms = timer(lambda: g.run(np.full(sweeps, w["T"]), w["refresh_interval"]))
        if best is None or ms < best[0]:
            best = (ms, nw)
    g.close()
    return {"flips_per_ns": updates(L, S, R, sweeps) / (best[0] * 1e6), "sweeps": sweeps,
            "words_per_thread": best[1], "us_per_sweep": 1e3 * best[0] / sweeps}


def leg_paper_shape(micsa, timer, stream, peaks, L=160, R=128, sweeps=400):
    """L = 160, 128 replicas of one sample, T = 0.7, refresh every 10."""
    out = {"L": L, "replicas": R, "sweeps": sweeps, "T": 0.7, "refresh_interval": 10}
    sched = np.full(sweeps, 0.7)
    g = micsa.Micsa(L, 1, R, 9, stream=stream)
    g.set_engine("multispin_global")
    out["multispin_launch"] = tune_planes(g, timer, sweeps=60)
    g.reinit(10)
    g.run(sched, 10)  # as long as the timed run: table sized, graph captured
    ms = timer(lambda: g.run(sched, 10))
    out["multispin_flips_per_ns"] = updates(L, 1, R, sweeps) / (ms * 1e6)
    out["multispin_ns_per_sweep"] = 1e6 * ms / sweeps
    out["multispin_roofline"] = plane_roofline(micsa, timer, stream, g, peaks)
    # the RNG-per-update Metropolis on the same bit planes (one uniform per site and
    # sweep from the same Philox counters): the paper's own comparison at this shape
    n_m = max(10, sweeps // 4)
    g.run_metropolis(np.full(n_m, 0.7))  # as long as the timed run
    ms = timer(lambda: g.run_metropolis(np.full(n_m, 0.7)))
    out["metropolis_planes_flips_per_ns"] = updates(L, 1, R, n_m) / (ms * 1e6)
    g.set_engine("stream")
    g.set_launch_config(4, 128, -1, True, 64)
    g.reinit(10)
    n_s = max(10, sweeps // 4)
    g.run(sched[:n_s], 10)
    ms = timer(lambda: g.run(sched[:n_s], 10))
    out["stream_flips_per_ns"] = updates(L, 1, R, n_s) / (ms * 1e6)
    nw = g.launch_config()["words_per_thread"]
    g.close()
    # one walker per spin (gamma = 1) wandering along +x after every timestep, refreshed on the
    # paper's log schedule t = 2^s - 1 (Sec. 2.6, 2.8): the configuration of the paper's timings
    gw = micsa.Micsa(L, 1, R, 11, stream=stream, walkers=True)
    gw.set_engine("multispin_global")
    gw.set_launch_config(out["multispin_launch"]["words_per_thread"], 128, -1, True, 64)
    gw.run_logrefresh(np.full(256, 0.7))
    ms = timer(lambda: gw.run_logrefresh(np.full(256, 0.7)))
    gw.close()
    out["walkers_log_refresh_flips_per_ns"] = updates(L, 1, R, 256) / (ms * 1e6)
    out["walkers_ns_per_timestep"] = 1e6 * ms / 256
    # six walker families (a timestep is six sweeps, family alpha wanders along
    # direction alpha), the paper's best-performing variant (Sec. 3)
    g6 = micsa.Micsa(L, 1, R, 12, stream=stream, gamma=6, walkers=True)
    g6.set_engine("multispin_global")
    g6.set_launch_config(out["multispin_launch"]["words_per_thread"], 128, -1, True, 64)
    # (runs of 128 timesteps: each run converts the state to bit planes and back once)
    g6.run_logrefresh(np.full(128, 0.7))
    ms = timer(lambda: g6.run_logrefresh(np.full(128, 0.7)))
    g6.close()
    out["walkers_gamma6_flips_per_ns"] = updates(L, 1, R, 128 * 6) / (ms * 1e6)
    out["micsa_over_metropolis_planes"] = {
        "daemons_refresh_10": out["multispin_flips_per_ns"] / out["metropolis_planes_flips_per_ns"],
        "one_walker_log_refresh": out["walkers_log_refresh_flips_per_ns"] / out["metropolis_planes_flips_per_ns"],
        "paper_h100_walkers_vs_metropolis": 1.9}
    out["paper_h100_walkers_total_ns_per_sweep"] = 121554 + 97378
    out["paper_h100_spin_update_kernel_ns_per_sweep"] = 121554
    out["paper_h100_flips_per_ns"] = 128 * 160 ** 3 / 121554.0
    return out


def leg_kstar(micsa, L=64, S=16, R=2, T=0.7, t_max=4096, gamma=6, stream=None):
    """Same-GPU Metropolis against MicSA with gamma walkers per spin on the same
    synthetic samples (couplings and starts from one seed) at T = 0.7: the energy
    per spin and the coherence length xi_12 (from C4 averaged over the samples, the
    integrals cut at three standard errors)
    on a log time grid, and the factor k with y_MicSA(t) = y_Metropolis(k t) for
    each, t in sweeps for Metropolis and in timesteps of gamma sweeps for MicSA
    (the paper's k*, from xi_12, is 6.034 for six walkers at T = 0.7)."""
    from paper_2506_16240_gb300 import analysis
    grid = sorted({int(round(10 ** (x / 10))) for x in range(0, int(10 * np.log10(t_max)) + 1)})
    N = L ** 3

    def curve(g, run, times):
        e_out, xi_out, t_prev = [], [], 0
        for tm in times:
            if tm > t_prev:
                run(g, tm - t_prev)
                t_prev = tm
            e, _, _ = g.measure()
            e_out.append(float(e.mean()) / N)
            xi_out.append(analysis.xi_of_samples(g.c4()))
        return np.array(e_out), np.array(xi_out)

    gm = micsa.Micsa(L, S, R, 21, stream=stream)
    e_met, xi_met = curve(gm, lambda g, n: g.run_metropolis(np.full(n, T)), grid)
    c4m = gm.c4()
    ratio_met = analysis.xi_of_samples(c4m, 2) / analysis.xi_of_samples(c4m, 1)  # xi_23 / xi_12 at the end
    gm.close()
    gw = micsa.Micsa(L, S, R, 21, stream=stream, gamma=gamma, walkers=True)
    gw.set_engine("multispin_global")
    grid_w = [t for t in grid if t <= t_max // 3]
    e_mic, xi_mic = curve(gw, lambda g, n: g.run_logrefresh(np.full(n, T)), grid_w)
    c4w = gw.c4()
    ratio_mic = analysis.xi_of_samples(c4w, 2) / analysis.xi_of_samples(c4w, 1)
    gw.close()
    tg, tw = np.array(grid, np.float64), np.array(grid_w, np.float64)
    sel = tw >= 16  # the refreshes at t = 2^s - 1 perturb the early energies
    k, mis, npts = analysis.fit_time_rescaling(tg, e_met, tw[sel], e_mic[sel], k_range=(1, 30))
    kx, misx, nx = analysis.fit_time_rescaling(tg, xi_met, tw[sel], xi_mic[sel], k_range=(1, 30))
    return {"k_star_energy": k, "rms_mismatch": float(np.sqrt(mis)), "points": npts,
            "k_star_xi12": kx, "rms_mismatch_xi12": float(np.sqrt(misx)), "points_xi12": nx, "gamma": gamma,
            "xi23_over_xi12_final": {"metropolis": ratio_met, "micsa": ratio_mic},
            "workload": f"L={L}, {S} samples x {R} replicas, T={T}: Metropolis to {t_max} sweeps, "
                        f"MicSA with {gamma} walkers per spin (log refresh) to {grid_w[-1]} timesteps",
            "paper_k_star_xi12": 6.034,
            "e_metropolis": [[t, round(v, 6)] for t, v in zip(grid, e_met)][::3],
            "e_micsa": [[t, round(v, 6)] for t, v in zip(grid_w, e_mic)][::3],
            "xi12_metropolis": [[t, round(v, 4)] for t, v in zip(grid, xi_met)][::3],
            "xi12_micsa": [[t, round(v, 4)] for t, v in zip(grid_w, xi_mic)][::3]}


def leg_metropolis(micsa, timer, stream, choice=None, n=10_000):
    """Same lattice under the RNG-per-update Metropolis kernel, in the fastest of a
    few launch shapes for that kernel, next to MicSA in the benchmark's tuned shape."""
    from paper_2506_16240_gb300 import autotune
    w = WORKLOAD
    T = w["T"]
    g = micsa.Micsa(w["L"], 1, w["replicas"], 3, stream=stream)
    shapes = []
    # (words per thread, block, replica chains, grid: -1 grid-stride, 0 one chunk per thread)
    for nw, blk, ch, bps in [(4, 128, 2, -1), (4, 128, 1, -1), (2, 128, 2, -1), (4, 256, 2, -1), (2, 256, 1, -1),
                             (4, 128, 2, 0), (4, 160, 2, 0), (2, 128, 2, 0)]:
        g.set_launch_config(nw, blk, bps, True, 64)
        g.set_replica_chains(ch)
        g.run_metropolis(np.full(1000, T))
        shapes.append((timer(lambda: g.run_metropolis(np.full(1000, T))), nw, blk, ch, bps))
    _, nw, blk, ch, bps = min(shapes)
    g.set_launch_config(nw, blk, bps, True, 64)
    g.set_replica_chains(ch)
    g.reinit(3)
    # warm-ups as long as the timed runs: sweep table sized, graphs captured (setup costs)
    g.run_metropolis(np.full(n, T))
    ms_metro = timer(lambda: g.run_metropolis(np.full(n, T)))
    if choice is not None:
        autotune.apply(g, choice)
    g.reinit(3)
    g.run(np.full(n, T), w["refresh_interval"])
    ms_micsa = timer(lambda: g.run(np.full(n, T), w["refresh_interval"]))
    g.close()
    u = updates(w["L"], 1, w["replicas"], n)
    return {"value": u / (ms_metro * 1e6), "unit": METRIC, "sweeps": n,
            "metropolis_launch": {"words_per_thread": nw, "block": blk, "replica_chains": ch, "blocks_per_sm": bps},
            "micsa_same_lattice": u / (ms_micsa * 1e6), "micsa_over_metropolis": ms_metro / ms_micsa}


def leg_quench_l32(micsa, timer, stream):
    from paper_2506_16240_gb300 import analysis
    L, S, R, T, n, r = 32, 64, 2, 0.7, 10_000, 10
    N = L ** 3
    grid = sorted(set([0] + [int(10 ** (k / 8)) for k in range(0, 33)]))
    g = micsa.Micsa(L, S, R, 2, stream=stream)
    from paper_2506_16240_gb300 import autotune
    tuned = autotune.tune(g, __import__("torch"), stream, sweeps=200, use_cache=False)
    g.reinit(2)
    series, t_prev, total_ms = [], 0, 0.0
    for tm in grid:
        if tm > t_prev:
            total_ms += timer(lambda: g.run(np.full(tm - t_prev, T), r))
            t_prev = tm
        e, a, q = g.measure()
        xi12 = analysis.xi_of_samples(g.c4()) if tm > 0 else 0.0  # outside the timed runs
        series.append((tm, float(e.mean() / N), float(((q / N) ** 2).mean()), xi12))
    eng = g.engine()
    c4 = g.c4().mean(axis=0)  # four-point correlation at t = 1e4, averaged over samples
    g.close()
    return {"value": updates(L, S, R, n) / (total_ms * 1e6), "unit": METRIC, "engine": eng, "launch": tuned,
            "c4_final": [round(float(v), 6) for v in c4[: L // 2 + 1]],
            "workload": "L=32, 64 samples x 2 replicas, T=0.7, 1e4 sweeps, refresh every 10",
            "e_final": series[-1][1], "q2_final": series[-1][2], "xi12_final": series[-1][3],
            "e_q2_xi12_vs_t": [[t, round(e, 6), round(q2, 8), round(x, 4)] for t, e, q2, x in series[::4]]
            + [list(series[-1])]}


def c4_instances():
    rng = np.random.default_rng(4)
    Ls = rng.choice([16, 24, 32, 48, 64], 256)
    rs = rng.integers(5, 21, 256)
    seeds = rng.integers(1, 2 ** 62, 256)
    return [(int(L), int(r), int(s)) for L, r, s in zip(Ls, rs, seeds)]


def pool_job_path(L, R, planes_budget):
    """Which part of a pool tick advances a job (the pool's own rules, bit-plane
    path on): 'smem' (L <= 32: the shared-memory multispin kernel), 'smem_planes'
    (L > 32 with one replica's six bit planes within the shared-memory budget; rows
    of 4 ceil(L/8) words), 'planes' (the other L > 32: global bit planes)."""
    if L <= 32:
        return "smem"
    WP = L * ((L + 31) // 32) * 4 * ((L // 2 + 3) // 4)
    return "smem_planes" if planes_budget and 6 * 4 * WP <= planes_budget else "planes"


def pool_roofline(jobs, seconds, K, planes_budget, peaks):
    """Algorithmic bytes per second of a pool run against the HBM peak. Per site
    update: byte streaming 5 + 1/R B (spin and daemon read and written, the
    opposite spin, the bond byte shared by R replicas); global bit planes
    (7 + 6/R) / 8 B; shared memory (both kernels): the state in and out once per
    tick, (4 + 1/R) / K B. jobs: (L, R, sweeps run)."""
    per_path, total_bytes, total_upd = {}, 0.0, 0
    for L, R, n in jobs:
        path = pool_job_path(L, R, planes_budget)
        b = {"bytes": 5 + 1 / R, "planes": (7 + 6 / R) / 8}.get(path, (4 + 1 / R) / K)
        upd = L ** 3 * R * n
        total_bytes += b * upd
        total_upd += upd
        per_path[path] = per_path.get(path, 0) + upd
    hbm = peaks.get("hbm_gbs") or 6800.0
    achieved = total_bytes / seconds / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
            "bytes_per_update": total_bytes / total_upd,
            "updates_by_path": {k: v / total_upd for k, v in per_path.items()},
            "note": "most updates run in shared memory (state in and out once per tick): far below the HBM "
                    "roofline, bound by integer/logic issue"}


def leg_batched(micsa, torch, stream, peaks, n_sweeps=20_000, loop_sweeps=2_000):
    from paper_2506_16240_gb300 import autotune
    inst = c4_instances()
    total = sum(updates(L, 1, 2, n_sweeps) for L, _, _ in inst)
    jobs = [(L, 2, s, n_sweeps, r, 2.5, 0.5) for L, r, s in inst]
    # pool shape (words per thread, chains, grid, shared-memory setting) from the autotuner,
    # on a scratch pool of the same jobs, for two tick lengths (the shared-memory path moves
    # a job's state in and out once per tick); the faster per sweep is kept
    best = None
    for K in (256, 1024):
        c = autotune.tune_pool_for_jobs(lambda: micsa.Pool(8 << 30, 512, K), jobs, ticks=1)
        if best is None or c["s_per_tick"] / K < best[0]["s_per_tick"] / best[1]:
            best = (c, K)
    choice, K = best
    choice = dict(choice, tick_sweeps=K)
    with micsa.Pool(8 << 30, 512, K) as p:
        autotune.apply_pool(p, choice)
        budget = p.smem_planes()[0]
        ids = [p.submit(*j) for j in jobs]
        assert all(i is not None for i in ids)
        p.wait()
        launches0 = p.stats()["launches"]
        t0 = time.perf_counter()
        left = set(ids)
        while left:
            p.tick()
            p.wait_ticks(2)
            for j in p.finished():
                p.poll(j, best_spins=False)
                left.discard(j)
        dt_pool = time.perf_counter() - t0
        launches = p.stats()["launches"] - launches0
    # the plain per-lattice launch loop (one handle per lattice, run back to back),
    # timed on the first loop_sweeps sweeps of the same schedule
    hs = [micsa.Micsa(L, 1, 2, s, stream=stream) for L, _, s in inst]
    sched = micsa.linear_schedule(2.5, 0.5, n_sweeps)[:loop_sweeps]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, (L, r, _) in zip(hs, inst):
        h.run(sched, r)
    torch.cuda.synchronize()
    dt_loop = time.perf_counter() - t0
    loop_upd = sum(updates(L, 1, 2, loop_sweeps) for L, _, _ in inst)
    for h in hs:
        h.close()
    batched, loop = total / (dt_pool * 1e9), loop_upd / (dt_loop * 1e9)
    return {"value": batched, "unit": METRIC, "per_lattice_loop": loop, "speedup": batched / loop,
            "wall_s": dt_pool, "launches": launches, "launch": choice,
            "roofline": pool_roofline([(L, 2, n_sweeps) for L, _, _ in inst], dt_pool, K, budget, peaks),
            "workload": "256 lattices L in {16,24,32,48,64} x 2 replicas, anneal 2.5->0.5 over 2e4 sweeps, "
                        "refresh 5..20; the loop is timed on its first 2e3 sweeps"}


def leg_serving(micsa, torch, stream, n_jobs, peaks, n_cap=600, slots=256, K=128):
    """The serving stream through the continuous-batching pool. Saturated capacity:
    n_cap requests of the same mix queued at once, more than the pool's slots, so
    that the pool stays full until the queue empties; the capacity is the attempts
    run in that window over its length. The Poisson stream of n_jobs is then
    offered at ~80% of that capacity (p50/p99 latency, aggregate rate)."""
    from paper_2506_16240_gb300 import autotune, serve
    cap_reqs = serve.poisson_stream(n_cap, 1e6, seed=55)
    desc = [(r.L, r.n_replicas, r.seed, r.n_sweeps, r.refresh_interval, r.T_start, r.T_end) for r in cap_reqs[:slots]]
    # tuned at the serving pool's own tick length: the shared-memory path moves a job's
    # state in and out once per tick, so shorter ticks would understate it
    choice = autotune.tune_pool_for_jobs(lambda: micsa.Pool(16 << 30, slots, K), desc)
    with micsa.Pool(16 << 30, slots, K) as p:
        autotune.apply_pool(p, choice)
        budget = p.smem_planes()[0]
        srv = serve.Server(p)
        l0 = p.stats()["launches"]
        srv.serve(cap_reqs, realtime=False)
        cap_launches = p.stats()["launches"] - l0
        sat_flips, sat_s = srv.saturated
        capacity = sat_flips / sat_s  # updates/s with the pool full
        drained = sum(r.updates for r in cap_reqs) / srv.wall  # the whole run, queue and tail included
    # the plain per-job loop: one handle per job, run one after another (first 64 jobs of the mix)
    loop_reqs = cap_reqs[:64]
    sched_cache = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in loop_reqs:
        key = (r.n_sweeps, r.T_start, r.T_end)
        if key not in sched_cache:
            sched_cache[key] = micsa.linear_schedule(r.T_start, r.T_end, r.n_sweeps)
        with micsa.Micsa(r.L, 1, r.n_replicas, r.seed, stream=stream) as h:
            h.run(sched_cache[key], r.refresh_interval)
            h.measure()
    loop_rate = sum(r.updates for r in loop_reqs) / (time.perf_counter() - t0)
    # Poisson stream offered at ~80% of the saturated capacity
    rate_hz = 0.8 * capacity / serve.mean_job_updates()
    reqs = serve.poisson_stream(n_jobs, rate_hz, seed=5)
    with micsa.Pool(16 << 30, slots, K) as p:
        autotune.apply_pool(p, choice)
        server = serve.Server(p)
        done = server.serve(reqs, realtime=True)
    out = serve.summarize(done, server.wall)
    out.update({"unit": METRIC, "arrival_rate_hz": rate_hz, "launch": choice, "slots": slots, "tick_sweeps": K,
                "roofline": pool_roofline([(r.L, r.n_replicas, r.n_sweeps) for r in done], server.wall, K, budget, peaks),
                "saturated_pool_flips_per_ns": capacity / 1e9, "saturated_window_s": sat_s,
                "capacity_run_flips_per_ns": drained / 1e9, "capacity_run_launches": cap_launches,
                "per_job_loop_flips_per_ns": loop_rate / 1e9, "saturated_over_loop": capacity / loop_rate,
                "workload": f"{n_jobs} Poisson jobs: L even 16..96, sweeps log-uniform 1e3..1e5, "
                            "1..4 replicas, anneal 3.0->0.3, refresh every 10; capacity on "
                            f"{n_cap} jobs of the same mix queued at once ({slots} slots), "
                            "the loop on 64 of them"})
    return out


# ------------------------------------------------------ profile cases --
# Small fixed workloads for ncu captures of the main kernels (`--profile-case
# NAME`): a few milliseconds of GPU work on a few tens of MB each, sized for
# `ncu --set full -k <kernel> -c <n>` captures that end by themselves.
#   stream        L=160, 1 x 2: 30 MicSA + 4 Metropolis sweeps
#   chains        the same lattice with the two replicas as two chains, 140 sweeps
#   single        the same with both replicas in each launch (one chain)
#   chains_l320, chains_l400  as chains at L = 320 (164 MB of state) and L = 400 (320 MB)
#   chains_bps0, chains_l400_bps0  as chains and chains_l400 with one thread per chunk (no
#                 grid-stride loop); chains_bps0_b96 / _b160 / _b192 / _b224 the same in
#                 blocks of 96, 160, 192, 224; chains_l400_b160, chains_l400_bps0_b160 at L = 400
#   multispin     L=32, 64 x 2: 128 sweeps, blocks of 64
#   planes        L=160, 1 x 128, bit planes: 12 sweeps
#   planes_r2     L=160, 1 x 2 (the headline lattice), bit planes: 24 sweeps
#   planes_metro  the L=160 x 128 lattice, 12 Metropolis sweeps
#   onchip        L=160, 1 x 2, on-chip engine: 2 x 64 sweeps
#   tma           L=160, 1 x 2, TMA engine: 12 sweeps
#   pool          64 mixed jobs, 2 ticks of 64 sweeps
#   batched       the 256 batched lattices in one pool, 2 ticks of 32 sweeps
#   plane_jobs_smem, plane_jobs_global  16 bit-plane jobs (L = 64 and 48), one tick of
#                 64 sweeps, in shared memory or on the global bit planes
#   plane_jobs_smem_norefresh  the same in shared memory with one refresh (t = 0)
def _micsa():
    import paper_2506_16240_gb300
    return paper_2506_16240_gb300


def case_stream():
    g = _micsa().Micsa(160, 1, 2, 3)
    g.set_engine("stream")
    g.run(np.full(30, 0.7), 10)
    g.run_metropolis(np.full(4, 0.7))
    return g.measure()[0]


def case_chains(L=160, chains=2, bps=-1, block=128):
    g = _micsa().Micsa(L, 1, 2, 3)
    g.set_engine("stream")
    g.set_launch_config(4, block, bps, True, 64)
    g.set_replica_chains(chains)
    g.run(np.full(140, 0.7), 10)  # 2 graph replays of 64 sweeps + 12 direct
    return g.measure()[0]


def case_planes():
    g = _micsa().Micsa(160, 1, 128, 3)
    g.set_engine("multispin_global")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run(np.full(12, 0.7), 10)
    return g.measure()[0][:4]


def case_planes_r2():
    g = _micsa().Micsa(160, 1, 2, 3)
    g.set_engine("multispin_global")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run(np.full(24, 0.7), 10)
    return g.measure()[0]


def case_planes_metro():
    g = _micsa().Micsa(160, 1, 128, 3)
    g.set_engine("multispin_global")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run_metropolis(np.full(12, 0.7))
    return g.measure()[0][:4]


def case_onchip():
    g = _micsa().Micsa(160, 1, 2, 3)
    g.set_launch_config(4, 128, -1, True, 64)
    g.set_engine("onchip", 64)
    g.run(np.full(128, 0.7), 10)
    return g.measure()[0]


def case_tma():
    g = _micsa().Micsa(160, 1, 2, 3)
    g.set_engine("tma")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run(np.full(12, 0.7), 10)
    return g.measure()[0]


def case_multispin():
    g = _micsa().Micsa(32, 64, 2, 2)
    g.set_engine("multispin", 64)
    g.run(np.full(128, 0.7), 10)
    return g.measure()[0][:4]


def case_pool():
    rng = np.random.default_rng(4)
    with _micsa().Pool(1 << 30, 128, 64) as p:
        ids = [p.submit(int(L), 2, int(s), 128, 10, 2.5, 0.5)
               for L, s in zip(rng.choice([16, 24, 32, 48, 64], 64), rng.integers(1, 2 ** 62, 64))]
        for _ in range(2):
            p.tick()
        p.wait()
        return [p.poll(j, best_spins=False)["energy"][0] for j in ids[:4]]


def case_batched(K=32, ticks=2):
    """The 256 batched lattices in one pool (default shape, the bit-plane jobs in
    shared memory in units of one replica: a 100 KB budget), ticks of K sweeps."""
    rng = np.random.default_rng(4)
    inst = zip(rng.choice([16, 24, 32, 48, 64], 256), rng.integers(5, 21, 256), rng.integers(1, 2 ** 62, 256))
    with _micsa().Pool(8 << 30, 512, K) as p:
        p.set_smem_planes(100 << 10, 1)
        ids = [p.submit(int(L), 2, int(s), 20_000, int(r), 2.5, 0.5) for L, r, s in inst]
        for _ in range(ticks):
            p.tick()
        p.wait()
        return len(ids), p.stats()["launches"]


def case_plane_jobs(smem=True, K=64, interval=10):
    """16 bit-plane jobs (8 of L = 64, 8 of L = 48, 2 replicas, refresh every
    `interval` sweeps) in one pool, one tick of K sweeps: the shared-memory kernel
    (smem, units of one replica) or the per-half-sweep launches over the global
    bit planes."""
    with _micsa().Pool(1 << 30, 64, K) as p:
        p.set_smem_planes((100 << 10) if smem else 0, 1)
        ids = [p.submit(L, 2, 100 + j, 10 * K, interval, 2.5, 0.5) for j, L in enumerate([64] * 8 + [48] * 8)]
        p.tick()
        p.wait()
        return len(ids), p.stats()["launches"]


def pool_breakdown(ticks=6, K=256):
    """Tick times of the batched workload's pool by content and shared-memory
    bit-plane setting (wall clock over `ticks` ticks after two untimed ones); one
    JSON line per row."""
    import time as _t
    micsa = _micsa()
    rng = np.random.default_rng(4)
    inst = [(int(L), int(r), int(s)) for L, r, s in
            zip(rng.choice([16, 24, 32, 48, 64], 256), rng.integers(5, 21, 256), rng.integers(1, 2 ** 62, 256))]
    rows = [("all", lambda L: True, (0, 1))]
    for cl in (False, True):
        for budget in (50 << 10, 100 << 10, 150 << 10):
            rows.append(("L >= 48", lambda L: L >= 48, (budget, 1, cl)))
        rows.append(("L >= 48", lambda L: L >= 48, (232432, 1, cl)))
    rows += [("all", lambda L: True, (100 << 10, 1, False)), ("all", lambda L: True, (150 << 10, 1, True)),
             ("all", lambda L: True, (50 << 10, 1, True)), ("L <= 32", lambda L: L <= 32, (0, 1))]
    for label, sel, smem in rows:
        with micsa.Pool(8 << 30, 512, K) as p:
            if smem is not None:
                p.set_smem_planes(*smem[:2])
                if len(smem) > 2:
                    p.set_smem_clusters(smem[2])
            for L, r, s in inst:
                if sel(L):
                    p.submit(L, 2, s, 10 ** 6, r, 2.5, 0.5)
            p.tick()
            p.tick()
            p.wait()
            t0 = _t.perf_counter()
            for _ in range(ticks):
                p.tick()
            p.wait()
            dt = (_t.perf_counter() - t0) / ticks
            upd = sum(L ** 3 * 2 for L, _, _ in inst if sel(L)) * K
            print(json.dumps({"jobs": label, "smem_planes": list(smem) if smem else "default (whole budget)",
                              "ms_per_tick": 1e3 * dt, "flips_per_ns": upd / (dt * 1e9)}))


PROFILE_CASES = {"stream": case_stream, "chains": case_chains, "multispin": case_multispin,
                 "single": lambda: case_chains(160, 1), "chains_l320": lambda: case_chains(320),
                 "chains_l400": lambda: case_chains(400), "batched": case_batched,
                 "chains_bps0_b160": lambda: case_chains(160, 2, 0, 160), "chains_bps0_b96": lambda: case_chains(160, 2, 0, 96), "chains_bps0_b192": lambda: case_chains(160, 2, 0, 192), "chains_bps0_b224": lambda: case_chains(160, 2, 0, 224), "chains_l400_b160": lambda: case_chains(400, 2, -1, 160), "chains_l400_bps0_b160": lambda: case_chains(400, 2, 0, 160), "chains_bps0": lambda: case_chains(160, 2, 0), "chains_l400_bps0": lambda: case_chains(400, 2, 0),
                 "plane_jobs_smem": case_plane_jobs, "plane_jobs_global": lambda: case_plane_jobs(False),
                 "plane_jobs_smem_norefresh": lambda: case_plane_jobs(True, interval=1 << 20),
                 "planes": case_planes, "planes_r2": case_planes_r2, "planes_metro": case_planes_metro, "onchip": case_onchip,
                 "tma": case_tma, "pool": case_pool}


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        print(args.profile_case, PROFILE_CASES[args.profile_case]())
        return 0
    if args.pool_breakdown:
        pool_breakdown()
        return 0
    if args.source_digests:
        print(json.dumps({k: kernel_digest(k) for k in KERNEL_SOURCES}))
        return 0

    import torch
    import paper_2506_16240_gb300 as micsa

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def gathered(x):
        return gather_ms(torch, x, rank, world, dev)

    w = WORKLOAD
    L, S, R = w["L"], w["samples"], w["replicas"]
    # a dedicated (non-default) stream: the library launches on it and the CUDA
    # events below are recorded on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    timer = Timer(torch, stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sched = np.full(args.sweeps, w["T"])
    seed = rank_seed(rank)
    g = micsa.Micsa(L, S, R, seed, stream=stream)
    from paper_2506_16240_gb300 import autotune
    # launch shape of the byte-layout engine for this lattice (int8 spins, uint8
    # daemons); the bit-plane engine is timed on the same workload in its own leg
    tuned = autotune.tune(g, torch, stream, use_cache=False, engines=("stream", "resident", "multispin", "onchip", "tma"))

    for k in range(args.warmup):
        g.reinit(seed + k)
        g.run(sched, w["refresh_interval"])
        g.measure()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms, launches, last_obs = [], 0, None
    for k in range(args.steps):
        flush.zero_()  # evict the previous step's lattice from L2 (512 MB > 129 MB)
        n0 = g.launch_count()

        def step():
            g.reinit(seed + 100 + k)
            g.run(sched, w["refresh_interval"])

        step_ms.append(timer(step))
        launches += g.launch_count() - n0
        last_obs = g.measure()
    barrier()
    clock_info = clocks.stop()
    value, total_ms = aggregate(world, gathered(sum(step_ms)), updates(L, S, R, args.sweeps) * args.steps)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    roofline = leg_roofline(micsa, timer, stream, L, peaks, choice=tuned)

    # -- end to end through the C ABI from pinned host buffers
    N = L ** 3
    J_host = torch.empty((S, N, 3), dtype=torch.int8, pin_memory=True).numpy()
    s_host = torch.empty((S, R, N), dtype=torch.int8, pin_memory=True).numpy()
    m_host = torch.zeros((S, R, N), dtype=torch.uint8, pin_memory=True).numpy()
    rng = np.random.default_rng(11 + rank)
    J_host[...] = rng.choice(np.array([-1, 1], np.int8), J_host.shape)
    s_host[...] = rng.choice(np.array([-1, 1], np.int8), s_host.shape)
    s_out = torch.empty((S, R, N), dtype=torch.int8, pin_memory=True).numpy()
    m_out = torch.empty((S, R, N), dtype=torch.uint8, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 2))
    import ctypes
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_couplings(J_host)
        g.set_state(s_host, m_host, 0)
        g.run(sched, w["refresh_interval"])
        g.measure()
        t_out = ctypes.c_int64()
        micsa._check(micsa.lib().micsa_get_state(g.h, s_out.ctypes.data_as(ctypes.c_void_p),
                                                 m_out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t_out)), g.h)
    torch.cuda.synchronize()
    e2e_value, _ = aggregate(world, gathered(1e3 * (time.perf_counter() - t0)),
                             updates(L, S, R, args.sweeps) * e2e_steps)
    e2e = {"value": e2e_value, "unit": METRIC,
           "h2d_bytes_per_step": int(J_host.nbytes + s_host.nbytes + m_host.nbytes),
           "d2h_bytes_per_step": int(s_out.nbytes + m_out.nbytes + 8 * (2 * S * R + S * R * (R - 1) // 2))}
    g.close()

    extras = {}
    if rank == 0 and not args.no_extras:
        legs = [("dram_point", lambda: leg_roofline(micsa, timer, stream, 400, peaks, n_plain=512, choice=tuned)),
                ("metropolis", lambda: leg_metropolis(micsa, timer, stream, choice=tuned)),
                ("quench_l32", lambda: leg_quench_l32(micsa, timer, stream)),
                ("batched", lambda: leg_batched(micsa, torch, stream, peaks)),
                ("serving", lambda: leg_serving(micsa, torch, stream, args.serving_jobs, peaks)),
                ("multispin_l160", lambda: leg_multispin_l160(micsa, timer, stream, peaks)),
                ("onchip_l160", lambda: leg_onchip_l160(micsa, timer, stream)),
                ("paper_shape", lambda: leg_paper_shape(micsa, timer, stream, peaks)),
                ("kstar", lambda: leg_kstar(micsa, stream=stream))]
        for name, fn in legs:
            try:
                extras[name] = fn()
            except Exception as exc:  # a failed side leg is reported, not hidden
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if rank == 0:
        e_last, _, q_last = last_obs
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": w["name"], "L": L, "samples": S, "replicas": R, "T": w["T"],
                       "sweeps_per_step": args.sweeps, "refresh_interval": w["refresh_interval"],
                       "parallelism": f"replicas{world}", "launch": tuned,
                       "l2": "flushed between steps (512 MB write); the 20.5 MB lattice stays L2-resident within a step"},
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "clocks": clock_info,
            "cpu_baseline": base,
            "final_energy_per_spin": [float(v) / N for v in e_last],
            "final_q2": [float(v / N) ** 2 for v in q_last],
        }
        out.update(extras)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
