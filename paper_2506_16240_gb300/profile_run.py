"""Small fixed workloads for profiler captures (ncu) of the main kernels.

    python -m paper_2506_16240_gb300.profile_run stream     # L=160, 1 x 2: 30 MicSA + 4 Metropolis sweeps
    python -m paper_2506_16240_gb300.profile_run chains     # the same with the two replicas as two chains
    python -m paper_2506_16240_gb300.profile_run multispin  # L=32, 64 x 2: 128 sweeps, blocks of 64
    python -m paper_2506_16240_gb300.profile_run planes     # L=160, 1 x 128, bit planes: 12 sweeps
    python -m paper_2506_16240_gb300.profile_run planes_metro  # the same lattice, 12 Metropolis sweeps
    python -m paper_2506_16240_gb300.profile_run onchip     # L=160, 1 x 2, on-chip engine: 2 x 64 sweeps
    python -m paper_2506_16240_gb300.profile_run tma        # L=160, 1 x 2, TMA engine: 12 sweeps
    python -m paper_2506_16240_gb300.profile_run pool       # 64 mixed jobs, 2 ticks of 64 sweeps

Each run is a few milliseconds of GPU work on a few tens of MB, sized for
`ncu --set full -k <kernel> -c <n>` captures that end by themselves.
"""
import sys

import numpy as np

import paper_2506_16240_gb300 as micsa


def stream():
    g = micsa.Micsa(160, 1, 2, 3)
    g.set_engine("stream")
    g.run(np.full(30, 0.7), 10)
    g.run_metropolis(np.full(4, 0.7))
    return g.measure()[0]


def chains():
    g = micsa.Micsa(160, 1, 2, 3)
    g.set_engine("stream")
    g.set_replica_chains(2)
    g.run(np.full(140, 0.7), 10)  # 2 graph replays of 64 sweeps + 12 direct
    return g.measure()[0]


def planes():
    g = micsa.Micsa(160, 1, 128, 3)
    g.set_engine("multispin_global")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run(np.full(12, 0.7), 10)
    return g.measure()[0][:4]


def planes_metro():
    g = micsa.Micsa(160, 1, 128, 3)
    g.set_engine("multispin_global")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run_metropolis(np.full(12, 0.7))
    return g.measure()[0][:4]


def onchip():
    g = micsa.Micsa(160, 1, 2, 3)
    g.set_launch_config(4, 128, -1, True, 64)
    g.set_engine("onchip", 64)
    g.run(np.full(128, 0.7), 10)
    return g.measure()[0]


def tma():
    g = micsa.Micsa(160, 1, 2, 3)
    g.set_engine("tma")
    g.set_launch_config(4, 128, -1, True, 0)  # direct launches
    g.run(np.full(12, 0.7), 10)
    return g.measure()[0]


def multispin():
    g = micsa.Micsa(32, 64, 2, 2)
    g.set_engine("multispin", 64)
    g.run(np.full(128, 0.7), 10)
    return g.measure()[0][:4]


def pool():
    rng = np.random.default_rng(4)
    with micsa.Pool(1 << 30, 128, 64) as p:
        ids = [p.submit(int(L), 2, int(s), 128, 10, 2.5, 0.5)
               for L, s in zip(rng.choice([16, 24, 32, 48, 64], 64), rng.integers(1, 2 ** 62, 64))]
        for _ in range(2):
            p.tick()
        p.wait()
        return [p.poll(j, best_spins=False)["energy"][0] for j in ids[:4]]


if __name__ == "__main__":
    mode = sys.argv[1] if len(sys.argv) > 1 else "stream"
    modes = {"stream": stream, "chains": chains, "multispin": multispin, "planes": planes,
             "planes_metro": planes_metro, "onchip": onchip,
             "tma": tma, "pool": pool}
    print(mode, modes[mode]())
