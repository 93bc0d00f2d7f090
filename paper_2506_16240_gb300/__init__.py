"""Python binding of ``libmicsa.so`` (include/micsa.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels; this module
converts numpy arrays / Python numbers to the C ABI and raises on error codes.
There is no CPU fallback: if the compiled library is missing the import of
:func:`lib` fails loudly.

Natural layout (as in the C ABI): ``site = (z*L + y)*L + x``; couplings
``J[S, N, 3]`` (+-1 for the +x, +y, +z bonds of each site), spins
``s[S, R, N]`` int8 +-1, daemons ``m[S, R, N]`` uint8 (energy 4m).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmicsa.so")

MICSA_OK = 0
MICSA_E_INVALID_ARG = -1
MICSA_E_OOM = -2
MICSA_E_CUDA = -3
MICSA_E_TIMEOUT = -4
MICSA_E_BUSY = -5
MICSA_E_NOT_FOUND = -6
MICSA_E_TOO_LARGE = -7
MICSA_ENGINE_AUTO, MICSA_ENGINE_STREAM, MICSA_ENGINE_RESIDENT, MICSA_ENGINE_MULTISPIN = 0, 1, 2, 3
MICSA_ENGINE_MULTISPIN_GLOBAL = 4
MICSA_ENGINE_ONCHIP = 5
MICSA_ENGINE_TMA = 6
ENGINES = {"auto": MICSA_ENGINE_AUTO, "stream": MICSA_ENGINE_STREAM, "resident": MICSA_ENGINE_RESIDENT,
           "multispin": MICSA_ENGINE_MULTISPIN, "multispin_global": MICSA_ENGINE_MULTISPIN_GLOBAL,
           "onchip": MICSA_ENGINE_ONCHIP, "tma": MICSA_ENGINE_TMA}
MICSA_NOALLOC_MAX_TERMS = 8192
MICSA_LAUNCH_REGCAP, MICSA_LAUNCH_PAIRS, MICSA_LAUNCH_REPS = 256, 512, 1024

_ERRNAMES = {-1: "MICSA_E_INVALID_ARG", -2: "MICSA_E_OOM", -3: "MICSA_E_CUDA",
             -4: "MICSA_E_TIMEOUT", -5: "MICSA_E_BUSY", -6: "MICSA_E_NOT_FOUND",
             -7: "MICSA_E_TOO_LARGE"}


class MicsaError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None

_c = ctypes
_P = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_ip = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); every symbol of include/micsa.h
SIGNATURES = {
    "micsa_create": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_uint64, ctypes.POINTER(_P)]),
    "micsa_create_ex": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_uint64,
                                   ctypes.POINTER(_P)]),
    "micsa_reinit": (_c.c_int, [_P, _c.c_uint64]),
    "micsa_set_couplings": (_c.c_int, [_P, _P]),
    "micsa_get_couplings": (_c.c_int, [_P, _P]),
    "micsa_run": (_c.c_int, [_P, _P, _c.c_int64, _c.c_int32]),
    "micsa_run_logrefresh": (_c.c_int, [_P, _P, _c.c_int64]),
    "micsa_run_metropolis": (_c.c_int, [_P, _P, _c.c_int64]),
    "micsa_measure": (_c.c_int, [_P, _P, _P, _P]),
    "micsa_correlation": (_c.c_int, [_P, _P]),
    "micsa_c4": (_c.c_int, [_P, _P]),
    "micsa_get_state": (_c.c_int, [_P, _P, _P, _i64p]),
    "micsa_set_state": (_c.c_int, [_P, _P, _P, _c.c_int64]),
    "micsa_set_stream": (_c.c_int, [_P, _P]),
    "micsa_sync": (_c.c_int, [_P]),
    "micsa_device_bytes": (_c.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "micsa_launch_count": (_c.c_int, [_P, _i64p]),
    "micsa_set_launch_config": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "micsa_get_launch_config": (_c.c_int, [_P, _ip, _ip, _ip, _ip, _ip]),
    "micsa_set_engine": (_c.c_int, [_P, _c.c_int, _c.c_int]),
    "micsa_get_engine": (_c.c_int, [_P, _ip]),
    "micsa_set_multispin_replicas": (_c.c_int, [_P, _c.c_int]),
    "micsa_wait_selftest": (_c.c_int, [_c.c_int64, _ip]),
    "micsa_set_replica_chains": (_c.c_int, [_P, _c.c_int]),
    "micsa_destroy": (None, [_P]),
    "micsa_last_error": (_c.c_char_p, [_P]),
    "micsa_measure_noalloc": (_c.c_int, [_P, _P, _P, _c.c_int, _c.c_int, _c.c_int, _P, _P, _P, _P]),
    "micsa_daemon_thresholds": (_c.c_int, [_c.c_double, _u64p]),
    "micsa_metro_thresholds": (_c.c_int, [_c.c_double, _u64p]),
}


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"` "
                "(there is no CPU fallback)")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(rc, h=None):
    if rc != MICSA_OK:
        msg = lib().micsa_last_error(h).decode() if h is not None else ""
        raise MicsaError(rc, msg)


def daemon_thresholds(T):
    th = (ctypes.c_uint64 * 3)()
    _check(lib().micsa_daemon_thresholds(float(T), th))
    return np.array(list(th), np.uint64)


def metro_thresholds(T):
    th = (ctypes.c_uint64 * 3)()
    _check(lib().micsa_metro_thresholds(float(T), th))
    return np.array(list(th), np.uint64)


def wait_selftest(polls=1000):
    """Run the on-chip engine's bounded wait on a flag nothing sets; True when
    it gave up and reported the time-out."""
    out = ctypes.c_int()
    _check(lib().micsa_wait_selftest(int(polls), ctypes.byref(out)))
    return bool(out.value)


def measure_noalloc(spins_ptr, daemons_ptr, J_ptr, L, n_samples, n_replicas, stream_ptr=None):
    """Observables of caller-owned device arrays (natural layout, raw device
    pointers as ints) through the allocation-free entry point; host results."""
    S, R = int(n_samples), int(n_replicas)
    e = np.zeros(S * R, np.int64)
    a = np.zeros(S * R, np.int64)
    q = np.zeros(S * R * (R - 1) // 2, np.int64)
    rc = lib().micsa_measure_noalloc(
        ctypes.c_void_p(spins_ptr), ctypes.c_void_p(daemons_ptr) if daemons_ptr else None,
        ctypes.c_void_p(J_ptr), int(L), S, R, _ptr(e), _ptr(a), _ptr(q) if q.size else None,
        ctypes.c_void_p(stream_ptr) if stream_ptr else None)
    if rc != MICSA_OK:
        raise MicsaError(rc, "micsa_measure_noalloc")
    return e, a, q


class Micsa:
    """One handle of the C ABI: S disorder samples x R replicas of an L^3 lattice."""

    def __init__(self, L, n_samples=1, n_replicas=2, seed=0, stream=None, gamma=1, walkers=False):
        self.L, self.S, self.R, self.seed = int(L), int(n_samples), int(n_replicas), int(seed)
        self.gamma, self.walkers = int(gamma), bool(walkers)
        self.N = self.L ** 3
        h = ctypes.c_void_p()
        if self.gamma == 1 and not self.walkers:
            rc = lib().micsa_create(self.L, self.S, self.R, ctypes.c_uint64(self.seed), ctypes.byref(h))
        else:
            rc = lib().micsa_create_ex(self.L, self.S, self.R, self.gamma, int(self.walkers),
                                       ctypes.c_uint64(self.seed), ctypes.byref(h))
        if rc != MICSA_OK:
            raise MicsaError(rc, f"micsa_create(L={L}, S={n_samples}, R={n_replicas})")
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "h", None):
            lib().micsa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer cudaStream_t, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().micsa_set_stream(self.h, ctypes.c_void_p(raw) if raw else None), self.h)

    def reinit(self, seed):
        """Redraw couplings and spins from `seed` on the device; t = 0."""
        self.seed = int(seed)
        _check(lib().micsa_reinit(self.h, ctypes.c_uint64(self.seed)), self.h)

    def set_couplings(self, J):
        J = np.ascontiguousarray(J, np.int8)
        assert J.size == self.S * self.N * 3
        _check(lib().micsa_set_couplings(self.h, _ptr(J)), self.h)

    def get_couplings(self):
        J = np.zeros((self.S, self.N, 3), np.int8)
        _check(lib().micsa_get_couplings(self.h, _ptr(J)), self.h)
        return J

    def run(self, schedule, refresh_interval):
        sched = np.ascontiguousarray(schedule, np.float64)
        _check(lib().micsa_run(self.h, _ptr(sched), len(sched), int(refresh_interval)), self.h)

    def run_logrefresh(self, schedule):
        sched = np.ascontiguousarray(schedule, np.float64)
        _check(lib().micsa_run_logrefresh(self.h, _ptr(sched), len(sched)), self.h)

    def run_metropolis(self, schedule):
        sched = np.ascontiguousarray(schedule, np.float64)
        _check(lib().micsa_run_metropolis(self.h, _ptr(sched), len(sched)), self.h)

    def measure(self):
        """(energy[S*R], aux[S*R], overlap[S*R(R-1)/2]) as int64 arrays."""
        e = np.zeros(self.S * self.R, np.int64)
        a = np.zeros(self.S * self.R, np.int64)
        q = np.zeros(self.S * self.R * (self.R - 1) // 2, np.int64)
        _check(lib().micsa_measure(self.h, _ptr(e), _ptr(a), _ptr(q) if q.size else None), self.h)
        return e, a, q

    def correlation(self):
        """G[S, L] integer sums of the four-point correlation (Sec. 3)."""
        G = np.zeros((self.S, self.L), np.int64)
        _check(lib().micsa_correlation(self.h, _ptr(G)), self.h)
        return G

    def c4(self):
        """C4[S, L]: the four-point correlation per sample (micsa_c4)."""
        C = np.zeros((self.S, self.L), np.float64)
        _check(lib().micsa_c4(self.h, _ptr(C)), self.h)
        return C

    def get_state(self):
        s = np.zeros((self.S, self.R, self.N), np.int8)
        m = np.zeros((self.S, self.R, self.N) if self.gamma == 1 else (self.S, self.R, self.gamma, self.N), np.uint8)
        t = ctypes.c_int64()
        _check(lib().micsa_get_state(self.h, _ptr(s), _ptr(m), ctypes.byref(t)), self.h)
        return s, m, t.value

    def set_state(self, spins=None, daemons=None, t=0):
        s = None if spins is None else np.ascontiguousarray(spins, np.int8)
        m = None if daemons is None else np.ascontiguousarray(daemons, np.uint8)
        _check(lib().micsa_set_state(self.h, _ptr(s), _ptr(m), int(t)), self.h)

    def sync(self):
        _check(lib().micsa_sync(self.h), self.h)

    def set_launch_config(self, words_per_thread=4, block=256, blocks_per_sm=-1, pdl=True,
                          graph_sweeps=64):
        _check(lib().micsa_set_launch_config(self.h, int(words_per_thread), int(block),
                                             int(blocks_per_sm), int(bool(pdl)), int(graph_sweeps)),
               self.h)

    def launch_config(self):
        v = [ctypes.c_int() for _ in range(5)]
        _check(lib().micsa_get_launch_config(self.h, *[ctypes.byref(x) for x in v]), self.h)
        keys = ("words_per_thread", "block", "blocks_per_sm", "pdl", "graph_sweeps")
        return {k: x.value for k, x in zip(keys, v)}

    def set_engine(self, engine="auto", resident_sweeps=None):
        """resident_sweeps: sweeps per launch of the resident, multispin and
        onchip engines (default 64, and 2048 for onchip)."""
        if resident_sweeps is None:
            resident_sweeps = 2048 if engine == "onchip" else 64
        _check(lib().micsa_set_engine(self.h, ENGINES[engine], int(resident_sweeps)), self.h)

    def set_replica_chains(self, chains=1):
        """Replica groups captured as concurrent kernel chains (1..4)."""
        _check(lib().micsa_set_replica_chains(self.h, int(chains)), self.h)

    def set_multispin_replicas(self, replicas_per_thread=0):
        """Replicas per thread of the multispin_global engine (0: automatic)."""
        _check(lib().micsa_set_multispin_replicas(self.h, int(replicas_per_thread)), self.h)

    def engine(self):
        v = ctypes.c_int()
        _check(lib().micsa_get_engine(self.h, ctypes.byref(v)), self.h)
        return {code: name for name, code in ENGINES.items()}[v.value]

    def launch_count(self):
        n = ctypes.c_int64()
        _check(lib().micsa_launch_count(self.h, ctypes.byref(n)), self.h)
        return n.value

    def device_bytes(self):
        n = ctypes.c_size_t()
        _check(lib().micsa_device_bytes(self.h, ctypes.byref(n)), self.h)
        return n.value


# ----------------------------------------------------------- batched pool --
MICSA_POOL_MAX_REPLICAS = 8


class JobDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_replicas", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("n_sweeps", ctypes.c_int64), ("refresh_interval", ctypes.c_int32),
                ("T_start", ctypes.c_double), ("T_end", ctypes.c_double)]


class JobResult(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_int64), ("sweeps_done", ctypes.c_int64),
                ("n_replicas", ctypes.c_int32),
                ("energy", ctypes.c_int64 * MICSA_POOL_MAX_REPLICAS),
                ("aux", ctypes.c_int64 * MICSA_POOL_MAX_REPLICAS),
                ("best_energy", ctypes.c_int64 * MICSA_POOL_MAX_REPLICAS),
                ("best_t", ctypes.c_int64 * MICSA_POOL_MAX_REPLICAS)]


SIGNATURES.update({
    "micsa_pool_create": (_c.c_int, [_c.c_size_t, _c.c_int, _c.c_int, ctypes.POINTER(_P)]),
    "micsa_pool_job_bytes": (_c.c_int, [ctypes.POINTER(JobDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "micsa_pool_submit": (_c.c_int, [_P, ctypes.POINTER(JobDesc), _i64p]),
    "micsa_pool_tick": (_c.c_int, [_P]),
    "micsa_pool_wait": (_c.c_int, [_P]),
    "micsa_pool_wait_ticks": (_c.c_int, [_P, _c.c_int]),
    "micsa_pool_poll": (_c.c_int, [_P, _c.c_int64, ctypes.POINTER(JobResult), _P]),
    "micsa_pool_poll_state": (_c.c_int, [_P, _c.c_int64, ctypes.POINTER(JobResult), _P, _P, _P]),
    "micsa_pool_stats": (_c.c_int, [_P, ctypes.POINTER(_c.c_int), ctypes.POINTER(ctypes.c_size_t), _i64p]),
    "micsa_pool_finished": (_c.c_int, [_P, _i64p, _c.c_int, ctypes.POINTER(_c.c_int)]),
    "micsa_pool_set_launch_config": (_c.c_int, [_P, _c.c_int, _c.c_int, _c.c_int]),
    "micsa_pool_set_shape": (_c.c_int, [_P, _c.c_int, _c.c_int]),
    "micsa_pool_set_planes": (_c.c_int, [_P, _c.c_int]),
    "micsa_pool_set_smem_planes": (_c.c_int, [_P, _c.c_size_t, _c.c_int]),
    "micsa_pool_set_smem_clusters": (_c.c_int, [_P, _c.c_int]),
    "micsa_pool_set_small_planes": (_c.c_int, [_P, _c.c_int]),
    "micsa_pool_get_smem_planes": (_c.c_int, [_P, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                              ctypes.POINTER(_c.c_int)]),
    "micsa_pool_last_error": (_c.c_char_p, [_P]),
    "micsa_pool_destroy": (None, [_P]),
})


def linear_schedule(T_start, T_end, n_sweeps):
    """T(k) exactly as the pool computes it: T0 + (T1 - T0) * (k / (n - 1))."""
    k = np.arange(n_sweeps, dtype=np.float64)
    if n_sweeps <= 1:
        return np.full(n_sweeps, float(T_start))
    return float(T_start) + (float(T_end) - float(T_start)) * (k / float(n_sweeps - 1))


class Pool:
    """Resident pool of annealing jobs advanced together (continuous batching)."""

    def __init__(self, arena_bytes=1 << 30, max_jobs=1024, tick_sweeps=64):
        h = ctypes.c_void_p()
        rc = lib().micsa_pool_create(int(arena_bytes), int(max_jobs), int(tick_sweeps), ctypes.byref(h))
        if rc != MICSA_OK:
            raise MicsaError(rc, "micsa_pool_create")
        self.h = h
        self.tick_sweeps = int(tick_sweeps)
        self.jobs = {}  # id -> (L, R)

    def _check(self, rc):
        if rc != MICSA_OK:
            raise MicsaError(rc, lib().micsa_pool_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().micsa_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def job_bytes(L, n_replicas, n_sweeps, refresh_interval):
        d = JobDesc(int(L), int(n_replicas), 0, int(n_sweeps), int(refresh_interval), 1.0, 1.0)
        n = ctypes.c_size_t()
        _check(lib().micsa_pool_job_bytes(ctypes.byref(d), ctypes.byref(n)))
        return n.value

    def submit(self, L, n_replicas, seed, n_sweeps, refresh_interval, T_start, T_end):
        """Job id, or None when the pool has no slot or memory for it now."""
        d = JobDesc(int(L), int(n_replicas), ctypes.c_uint64(int(seed)).value, int(n_sweeps),
                    int(refresh_interval), float(T_start), float(T_end))
        jid = ctypes.c_int64()
        rc = lib().micsa_pool_submit(self.h, ctypes.byref(d), ctypes.byref(jid))
        if rc == MICSA_E_BUSY:
            return None
        self._check(rc)
        self.jobs[jid.value] = (int(L), int(n_replicas))
        return jid.value

    def tick(self):
        self._check(lib().micsa_pool_tick(self.h))

    def wait(self):
        self._check(lib().micsa_pool_wait(self.h))

    def wait_ticks(self, max_pending):
        self._check(lib().micsa_pool_wait_ticks(self.h, int(max_pending)))

    def poll(self, job_id, best_spins=True, final_state=False):
        """Result dict of a finished job (and frees it), or None while it runs.
        final_state: also the final spins and daemons [R, N] (natural layout)."""
        L, R = self.jobs[job_id]
        res = JobResult()
        spins = np.zeros((R, L ** 3), np.int8) if best_spins else None
        fs = np.zeros((R, L ** 3), np.int8) if final_state else None
        fm = np.zeros((R, L ** 3), np.uint8) if final_state else None
        rc = lib().micsa_pool_poll_state(self.h, int(job_id), ctypes.byref(res), _ptr(spins), _ptr(fs), _ptr(fm))
        if rc == MICSA_E_BUSY:
            return None
        self._check(rc)
        del self.jobs[job_id]
        out = {"job_id": res.job_id, "sweeps_done": res.sweeps_done,
               "energy": np.array(res.energy[:R], np.int64), "aux": np.array(res.aux[:R], np.int64),
               "best_energy": np.array(res.best_energy[:R], np.int64),
               "best_t": np.array(res.best_t[:R], np.int64)}
        if best_spins:
            out["best_spins"] = spins
        if final_state:
            out["spins"], out["daemons"] = fs, fm
        return out

    def finished(self, max_ids=4096):
        """Ids of finished jobs that can be polled now (non-blocking)."""
        ids = (ctypes.c_int64 * max_ids)()
        n = ctypes.c_int()
        self._check(lib().micsa_pool_finished(self.h, ids, int(max_ids), ctypes.byref(n)))
        return [ids[i] for i in range(n.value)]

    def stats(self):
        n = ctypes.c_int()
        free = ctypes.c_size_t()
        launches = ctypes.c_int64()
        self._check(lib().micsa_pool_stats(self.h, ctypes.byref(n), ctypes.byref(free), ctypes.byref(launches)))
        return {"live_jobs": n.value, "free_bytes": free.value, "launches": launches.value}

    def set_launch_config(self, blocks_per_sm, pdl=True, use_graph=True):
        self._check(lib().micsa_pool_set_launch_config(self.h, int(blocks_per_sm), int(bool(pdl)),
                                                       int(bool(use_graph))))

    def set_shape(self, max_words=4, chains=2):
        """Words per thread (cap 1, 2 or 4) and concurrent kernel chains (1..4) of
        the streaming jobs' half-sweeps; results do not depend on them."""
        self._check(lib().micsa_pool_set_shape(self.h, int(max_words), int(chains)))

    def set_smem_planes(self, smem_bytes, blocks_per_sm=1):
        """Shared-memory budget (bytes, 0: off) and grid of the persistent kernel that
        sweeps the bit-plane jobs admitted from now on in shared memory; results do
        not depend on it."""
        self._check(lib().micsa_pool_set_smem_planes(self.h, int(smem_bytes), int(blocks_per_sm)))

    def set_smem_clusters(self, on=True):
        """Split the shared-memory units of the jobs admitted from now on (32 < L <= 128)
        over thread-block clusters of one CTA per z word; results do not depend on it."""
        self._check(lib().micsa_pool_set_smem_clusters(self.h, int(bool(on))))

    def set_small_planes(self, on=True):
        """Jobs with L <= 32 admitted from now on as bit planes in shared memory (CTAs of
        128 threads) instead of the multispin kernel (the default, faster on such
        lattices); results do not depend on it."""
        self._check(lib().micsa_pool_set_small_planes(self.h, int(bool(on))))

    def smem_planes(self):
        """(budget bytes, the device's largest budget, blocks per SM) of the
        shared-memory bit-plane path."""
        b, m, n = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
        self._check(lib().micsa_pool_get_smem_planes(self.h, ctypes.byref(b), ctypes.byref(m), ctypes.byref(n)))
        return b.value, m.value, n.value

    def set_planes(self, on=True):
        """Bit-plane half-sweeps for the jobs admitted from now on with L above
        32; results do not depend on it."""
        self._check(lib().micsa_pool_set_planes(self.h, int(bool(on))))
