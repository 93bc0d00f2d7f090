"""Parity at the full sizes of the paper-shaped workloads, against stored values
written by ``tests/golden/make_golden.py`` from the CPU oracle alone.

  L = 32 quench: 64 samples x 2 replicas, T = 0.7, refresh every 10, all 10^4
      sweeps; H_EA and Q_ab at every point of the log time grid, final H_aux,
      final spins and daemons (SHA-256 of the natural-layout bytes).
  L = 160 quench (the benchmark lattice, seed 3): the first 10^3 sweeps; H_EA,
      H_aux and Q every 100 sweeps, spins and daemons at t = 100, 500, 1000.
  Batched: the first 16 of the 256 lattices of the batched workload, run in one
      pool together with the other 240 for all 2 x 10^4 sweeps; final H_EA,
      H_aux, spins and daemons of each.

Equal SHA-256 digests mean equal bytes, i.e. every spin and daemon equal.
"""
import hashlib
import os

import numpy as np
import pytest

import paper_2506_16240_gb300 as micsa

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _field(tokens, key, cast=int):
    """Values after `key` up to the next alphabetic key."""
    i = tokens.index(key) + 1
    out = []
    while i < len(tokens) and not tokens[i].isalpha():
        out.append(cast(tokens[i]))
        i += 1
    return out


def _quench_l32_golden():
    grid, E, Q, fin = [], {}, {}, {}
    for tok in _rows("quench_L32_64x2.txt"):
        if tok[0] == "t":
            t = int(tok[1])
            grid.append(t)
            E[t] = np.array(_field(tok, "E"), np.int64)
            Q[t] = np.array(_field(tok, "Q"), np.int64)
        else:
            fin[tok[0]] = tok[1:]
    return grid, E, Q, fin


@pytest.mark.parametrize("engine", ["auto", "stream", "multispin_global"])
def test_quench_l32_all_samples_all_sweeps_match_oracle(engine):
    grid, E, Q, fin = _quench_l32_golden()
    assert grid[-1] == 10_000 and len(E[0]) == 128 and len(Q[0]) == 64
    with micsa.Micsa(32, 64, 2, 2) as g:
        g.set_engine(engine)
        t_prev = 0
        for t in grid:
            if t > t_prev:
                g.run(np.full(t - t_prev, 0.7), 10)
                t_prev = t
            e, a, q = g.measure()
            np.testing.assert_array_equal(e, E[t], err_msg=f"{engine}: H_EA at t={t}")
            np.testing.assert_array_equal(q, Q[t], err_msg=f"{engine}: Q at t={t}")
        np.testing.assert_array_equal(a, np.array(fin["final_aux"], np.int64), err_msg=f"{engine}: final H_aux")
        s, m, t = g.get_state()
    assert t == 10_000
    assert sha(s) == fin["final_spins_sha256"][0], f"{engine}: final spins differ"
    assert sha(m) == fin["final_daemons_sha256"][0], f"{engine}: final daemons differ"


# launch shapes of the L = 160 lattice: the benchmark's tuned shape (two replica
# chains, 4 words per thread, blocks of 128, graph replays of 64 sweeps), direct
# launches, the bit planes in HBM, the TMA engine
L160_SHAPES = {
    "stream_chains": ("stream", (4, 128, -1, True, 64), 2),
    "stream_direct": ("stream", (2, 256, -1, True, 0), 1),
    "planes": ("multispin_global", (4, 128, -1, True, 64), 1),
    "tma": ("tma", (4, 128, -1, True, 64), 1),
}


@pytest.mark.parametrize("shape", sorted(L160_SHAPES))
def test_quench_l160_first_thousand_sweeps_match_oracle(shape):
    engine, lc, chains = L160_SHAPES[shape]
    rows = {int(tok[1]): tok for tok in _rows("quench_L160_1x2.txt")}
    assert sorted(rows) == list(range(100, 1001, 100))
    with micsa.Micsa(160, 1, 2, 3) as g:
        g.set_engine(engine)
        g.set_launch_config(*lc)
        g.set_replica_chains(chains)
        for t in range(100, 1001, 100):
            g.run(np.full(100, 0.7), 10)
            tok = rows[t]
            e, a, q = g.measure()
            np.testing.assert_array_equal(e, _field(tok, "E"), err_msg=f"{shape}: H_EA at t={t}")
            np.testing.assert_array_equal(a, _field(tok, "A"), err_msg=f"{shape}: H_aux at t={t}")
            np.testing.assert_array_equal(q, _field(tok, "Q"), err_msg=f"{shape}: Q at t={t}")
            if "S" in tok:
                s, m, tt = g.get_state()
                assert tt == t
                assert sha(s) == _field(tok, "S", str)[0], f"{shape}: spins differ at t={t}"
                assert sha(m) == _field(tok, "M", str)[0], f"{shape}: daemons differ at t={t}"


def _batched_instances():
    rng = np.random.default_rng(4)
    Ls = rng.choice([16, 24, 32, 48, 64], 256)
    rs = rng.integers(5, 21, 256)
    seeds = rng.integers(1, 2 ** 62, 256)
    return [(int(L), int(r), int(s)) for L, r, s in zip(Ls, rs, seeds)]


@pytest.mark.parametrize("shape", [None, (2, 3, 6)])
def test_batched_workload_subset_matches_oracle(shape):
    """All 256 lattices in one pool (ticks of 256 sweeps), as in the benchmark;
    shape: (words cap, chains, blocks per SM) of the pool, None for its default."""
    golden = {int(tok[1]): tok for tok in _rows("batched_subset16.txt")}
    inst = _batched_instances()
    n = 20_000
    with micsa.Pool(8 << 30, 512, 256) as p:
        if shape:
            p.set_shape(shape[0], shape[1])
            p.set_launch_config(shape[2])
        ids = [p.submit(L, 2, s, n, r, 2.5, 0.5) for L, r, s in inst]
        assert all(i is not None for i in ids)
        res = {}
        while len(res) < len(ids):
            p.tick()
            p.wait_ticks(2)
            for jid in p.finished():
                idx = ids.index(jid)
                res[idx] = p.poll(jid, best_spins=False, final_state=idx in golden)
    assert len(golden) == 16
    for idx, tok in golden.items():
        L, r, seed = inst[idx]
        assert (int(tok[3]), int(tok[5]), int(tok[7])) == (L, r, seed)
        what = f"job {idx} (L={L}, r={r})"
        assert res[idx]["sweeps_done"] == n
        np.testing.assert_array_equal(res[idx]["energy"], _field(tok, "E"), err_msg=what)
        np.testing.assert_array_equal(res[idx]["aux"], _field(tok, "A"), err_msg=what)
        assert sha(res[idx]["spins"]) == _field(tok, "S", str)[0], f"{what}: final spins differ"
        assert sha(res[idx]["daemons"]) == _field(tok, "M", str)[0], f"{what}: final daemons differ"
