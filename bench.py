#!/usr/bin/env python
"""Benchmark of the MicSA hot path on GB300 (one JSON line on rank 0).

Workload (one "step"): the single-lattice quench -- a 3D EA +-J lattice with
L = 160 (4,096,000 spins), 1 disorder sample x 2 replicas, couplings and a
random start drawn on the device from the step's seed, quenched to T = 0.7 for
10^5 MicSA sweeps with a daemon refresh every 10 sweeps, then the exact energy
and overlap are measured. Metric: spin-flip attempts per ns
(N x replicas x samples x sweeps / device time of the step).

Legs reported on the same JSON line:
  value       device time of the step (CUDA events on the launching stream),
              state resident in HBM, L2 flushed between steps
  e2e         the same job through the C ABI from pinned host buffers:
              couplings and initial spins copied in, final spins, daemons and
              observables copied out, all inside the timed region
  roofline    the plain half-sweep kernel: algorithmic bytes per launch over
              its average duration in a timed run of plain sweeps
  metropolis  the random-number-per-update Metropolis kernel on the same
              lattice (same layout), spin-flips/ns
  cpu_baseline the CPU oracle (single thread) on a bounded sample of sweeps

--impl reference times the oracle itself (the deliberately slow reference).
Multi-GPU (torchrun): one independent lattice per rank (weak scaling, no
data-path collective); the barrier and the max over ranks only time the job.
"""
import argparse
import json
import math
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--sweeps", type=int, default=WORKLOAD["sweeps"],
                    help="sweeps per step (profiling runs only; reported numbers use the default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def updates_per_step(sweeps):
    w = WORKLOAD
    return w["L"] ** 3 * w["samples"] * w["replicas"] * sweeps


# ------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
    """The oracle on the bench lattice for `sweeps` sweeps; returns (updates, seconds)."""
    import oracle
    w = WORKLOAD
    O = oracle.Oracle()
    st = O.create(w["L"], w["samples"], w["replicas"], seed)
    t0 = time.perf_counter()
    O.run(st, np.full(sweeps, w["T"]), w["refresh_interval"])
    dt = time.perf_counter() - t0
    return updates_per_step(sweeps), dt


def cpu_baseline(target_s=12.0):
    upd1, dt1 = oracle_sample(2)
    n = max(2, int(target_s / max(dt1 / 2, 1e-3)))
    n = min(n, 200)
    upd, dt = oracle_sample(n)
    return {"value": upd / (dt * 1e9), "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{n} sweeps of the L=160 1x2 lattice at T=0.7 (refresh every 10), "
                      f"single-threaded C oracle, {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOAD
    sweeps_per_step = 10
    for _ in range(args.warmup):
        oracle_sample(2)
    times = []
    for k in range(args.steps):
        upd, dt = oracle_sample(sweeps_per_step, seed=100 + k)
        times.append(dt)
    total_upd = updates_per_step(sweeps_per_step) * args.steps
    value = total_upd / (sum(times) * 1e9)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
        "data": "synthetic", "config": {"workload": w["name"], "L": w["L"], "samples": w["samples"],
                                        "replicas": w["replicas"],
                                        "sample_per_step": f"{sweeps_per_step} sweeps"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"{sweeps_per_step} sweeps per step of the L=160 1x2 lattice"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------- GPU --
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2506_16240_gb300 as micsa

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    w = WORKLOAD
    # a dedicated (non-default) stream: the library launches on it and the CUDA
    # events below are recorded on it
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    sched = np.full(args.sweeps, w["T"])
    base_seed = 3 + 1000 * rank  # independent lattice per rank
    g = micsa.Micsa(w["L"], w["samples"], w["replicas"], base_seed, stream=stream)

    def one_step(seed):
        g.reinit(seed)
        g.run(sched, w["refresh_interval"])
        return g.measure()  # synchronous: exact H, H_aux, overlap

    for k in range(args.warmup):
        one_step(base_seed + k)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    launches0 = g.launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    step_ms = []
    last_obs = None
    for k in range(args.steps):
        flush.zero_()  # evict the previous step's lattice from L2 (512 MB > 129 MB)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.reinit(base_seed + 100 + k)
        g.run(sched, w["refresh_interval"])
        ev1.record(stream)
        last_obs = g.measure()
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    barrier()
    clock_info = clocks.stop()
    launches = g.launch_count() - launches0 - args.steps  # measure kernels are outside the events
    total_ms = max_over_ranks(sum(step_ms))
    ms_per_step = total_ms / args.steps
    value = world * updates_per_step(args.sweeps) * args.steps / (total_ms * 1e6)

    # -- roofline of the plain half-sweep kernel: timed run without refreshes
    n_plain = 2000
    g.reinit(base_seed)
    g.run(np.full(1, w["T"]), w["refresh_interval"])  # t = 0 refresh
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.run(np.full(n_plain, w["T"]), 2 ** 31 - 1)  # t = 1 .. n_plain: no refresh
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1)
    launch_us = 1e3 * plain_ms / (2 * n_plain)
    L, R, S = w["L"], w["replicas"], w["samples"]
    half_sites = L ** 3 // 2 * S
    bytes_per_launch = half_sites * (5 * R + 1)  # s, m read+write per replica, bond, opposite spins
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    achieved = bytes_per_launch / (launch_us * 1e-6) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "kernel": "micsa::half_sweep_kernel<4,0> (plain MicSA half-sweep)",
                "bytes_per_launch": bytes_per_launch, "launch_us": launch_us,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # -- Metropolis on the same lattice and layout
    n_metro = 10_000
    g.reinit(base_seed)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.run_metropolis(np.full(n_metro, w["T"]))
    ev1.record(stream)
    torch.cuda.synchronize()
    metro_ms = ev0.elapsed_time(ev1)
    metro = {"value": updates_per_step(n_metro) / (metro_ms * 1e6), "unit": METRIC,
             "sweeps": n_metro, "ms": metro_ms}
    g.reinit(base_seed)
    g.run(np.full(n_metro, w["T"]), w["refresh_interval"])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    g.run(np.full(n_metro, w["T"]), w["refresh_interval"])
    ev1.record(stream)
    torch.cuda.synchronize()
    micsa_same_ms = ev0.elapsed_time(ev1)
    metro["micsa_same_sweeps_value"] = updates_per_step(n_metro) / (micsa_same_ms * 1e6)

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
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_couplings(J_host)
        g.set_state(s_host, m_host, 0)
        g.run(sched, w["refresh_interval"])
        e, a, q = g.measure()
        _lib = micsa.lib()
        import ctypes
        t_out = ctypes.c_int64()
        micsa._check(_lib.micsa_get_state(g.h, s_out.ctypes.data_as(ctypes.c_void_p),
                                          m_out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t_out)), g.h)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": world * updates_per_step(args.sweeps) * e2e_steps / (e2e_s * 1e9), "unit": METRIC,
           "h2d_bytes_per_step": int(J_host.nbytes + s_host.nbytes + m_host.nbytes),
           "d2h_bytes_per_step": int(s_out.nbytes + m_out.nbytes + 8 * (2 * S * R + S * R * (R - 1) // 2))}

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline()

    if rank == 0:
        e_last, a_last, q_last = last_obs
        out = {
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": w["name"], "L": L, "samples": S, "replicas": R, "T": w["T"],
                       "sweeps_per_step": args.sweeps, "refresh_interval": w["refresh_interval"],
                       "parallelism": f"replicas{world}",
                       "l2": "flushed between steps (512 MB write); the 20.5 MB lattice stays L2-resident within a step"},
            "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "clocks": clock_info,
            "metropolis": metro, "cpu_baseline": base,
            "final_energy_per_spin": [float(v) / N for v in e_last],
            "final_q2": [float(v / N) ** 2 for v in q_last],
        }
        print(json.dumps(out))
    g.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
