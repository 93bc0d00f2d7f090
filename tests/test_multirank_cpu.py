"""CPU (gloo) tests of the multi-rank host logic of bench.py: with N ranks each
rank runs its own lattice (weak scaling, no data-path collective); the job's
value is all ranks' updates over the slowest rank's time, and the reference
arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms = bench.gather_ms(torch, my_ms, rank, world, "cpu")
        value, total = bench.aggregate(world, ms, updates_per_rank=10 ** 9)
        q.put((rank, ms, value, total, bench.rank_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_aggregate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, v0, t0, s0), (r1, ms1, v1, t1, s1) = res
    assert ms0 == ms1 == [100.0, 150.0]
    assert t0 == t1 == 150.0
    # 2 ranks x 1e9 updates over 150 ms = 13.33 updates/ns
    assert v0 == v1 == pytest.approx(2 * 1e9 / (150.0 * 1e6))
    assert s0 != s1  # independent lattices


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_clock_parsing():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1950, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active"]
    c = bench.parse_clock_lines(lines)
    assert c["sm_mhz"] == 2010.0 and c["sm_max_mhz"] == 2070.0 and c["reasons"] == ["sw_power_cap"]
