"""ctypes front end of the plain-C MicSA oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. Arrays use the natural layout
``site = (z*L + y)*L + x``: couplings ``J[S, N, 3]`` (forward bonds +x, +y, +z,
values +-1), spins ``s[S, R, N]`` (int8 +-1), daemons ``m[S, R, N]`` (uint8,
energy 4m). See ``micsa_oracle.h`` for the paper passage each function follows.
"""
import ctypes
import numpy as np

from . import build as _build

_libs = {}

_i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_c_i64p = ctypes.POINTER(ctypes.c_int64)


def _declare(lib):
    c = ctypes
    sig = {
        "orc_philox4x32_10": (None, [_u32p, _u32p, _u32p]),
        "orc_daemon_thresholds": (c.c_int, [c.c_double, _u64p]),
        "orc_metro_thresholds": (c.c_int, [c.c_double, _u64p]),
        "orc_init_couplings": (None, [c.c_int, c.c_uint64, c.c_int64, _i8p]),
        "orc_init_spins": (None, [c.c_int, c.c_uint64, c.c_int64, _i8p]),
        "orc_energy": (c.c_int64, [c.c_int, _i8p, _i8p]),
        "orc_delta_h": (c.c_int, [c.c_int, _i8p, _i8p, c.c_int64]),
        "orc_refresh": (c.c_int, [c.c_int, c.c_uint64, c.c_int64, c.c_int64, c.c_double, _u8p]),
        "orc_half_sweep": (None, [c.c_int, _i8p, _i8p, _u8p, c.c_int]),
        "orc_serial_sweep": (None, [c.c_int, _i8p, _i8p, _u8p]),
        "orc_run": (c.c_int, [c.c_int, c.c_int, c.c_int, c.c_uint64, _i8p, _i8p, _u8p,
                              _c_i64p, _f64p, c.c_int64, c.c_int32, c.c_int]),
        "orc_run_logrefresh": (c.c_int, [c.c_int, c.c_int, c.c_int, c.c_uint64, _i8p, _i8p,
                                         _u8p, _c_i64p, _f64p, c.c_int64]),
        "orc_wander": (None, [c.c_int, _u8p, c.c_int, c.c_int]),
        "orc_run_ex": (c.c_int, [c.c_int, c.c_int, c.c_int, c.c_int, c.c_int, c.c_uint64, _i8p, _i8p,
                                 _u8p, _c_i64p, _f64p, c.c_int64, c.c_int32]),
        "orc_run_metropolis": (c.c_int, [c.c_int, c.c_int, c.c_int, c.c_uint64, _i8p, _i8p,
                                         _c_i64p, _f64p, c.c_int64, c.c_int]),
        "orc_measure": (None, [c.c_int, c.c_int, c.c_int, _i8p, _i8p, _u8p,
                               c.c_void_p, c.c_void_p, c.c_void_p]),
        "orc_correlation": (c.c_int, [c.c_int, c.c_int, c.c_int, _i8p, _i64p]),
        "orc_enumerate_dos": (c.c_int, [c.c_int, _i8p, _i64p]),
        "orc_all_energies": (c.c_int, [c.c_int, _i8p, _i64p]),
        "orc_l2_transition_micsa": (c.c_int, [_i8p, _f64p, _f64p]),
        "orc_l2_transition_metro": (c.c_int, [_i8p, c.c_double, _f64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args


def lib(mutant=0):
    if mutant not in _libs:
        handle = ctypes.CDLL(_build.build(mutant))
        _declare(handle)
        _libs[mutant] = handle
    return _libs[mutant]


class Oracle:
    """Thin wrapper over one build of the C oracle (``mutant`` > 0 plants a mistake)."""

    def __init__(self, mutant=0):
        self.lib = lib(mutant)

    # -- random numbers and thresholds -----------------------------------
    def philox(self, ctr, key):
        out = np.zeros(4, np.uint32)
        self.lib.orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
        return out

    def daemon_thresholds(self, T):
        th = np.zeros(3, np.uint64)
        if self.lib.orc_daemon_thresholds(float(T), th):
            raise ValueError(f"bad temperature {T}")
        return th

    def metro_thresholds(self, T):
        th = np.zeros(3, np.uint64)
        if self.lib.orc_metro_thresholds(float(T), th):
            raise ValueError(f"bad temperature {T}")
        return th

    # -- state -------------------------------------------------------------
    def couplings(self, L, seed, sample=0):
        J = np.zeros((L ** 3, 3), np.int8)
        self.lib.orc_init_couplings(L, seed, sample, J)
        return J

    def spins(self, L, seed, gid):
        s = np.zeros(L ** 3, np.int8)
        self.lib.orc_init_spins(L, seed, gid, s)
        return s

    def refresh(self, L, seed, gid, t, T):
        m = np.zeros(L ** 3, np.uint8)
        if self.lib.orc_refresh(L, seed, gid, t, float(T), m):
            raise ValueError("bad refresh arguments")
        return m

    def energy(self, L, J, s):
        return int(self.lib.orc_energy(L, np.ascontiguousarray(J, np.int8),
                                       np.ascontiguousarray(s, np.int8)))

    def delta_h(self, L, J, s, site):
        return int(self.lib.orc_delta_h(L, J, s, site))

    def half_sweep(self, L, J, s, m, parity):
        self.lib.orc_half_sweep(L, J, s, m, parity)

    def serial_sweep(self, L, J, s, m):
        self.lib.orc_serial_sweep(L, J, s, m)

    def create(self, L, S, R, seed, gamma=1, walkers=False):
        """Initial state of micsa_create: couplings and spins from the seed, t = 0.
        With gamma > 1 the daemons are m[S, R, gamma, N]."""
        N = L ** 3
        J = np.stack([self.couplings(L, seed, a) for a in range(S)])
        s = np.stack([self.spins(L, seed, g) for g in range(S * R)]).reshape(S, R, N)
        m = np.zeros((S, R, N) if gamma == 1 else (S, R, gamma, N), np.uint8)
        return {"L": L, "S": S, "R": R, "seed": seed, "J": J, "s": s, "m": m, "t": 0,
                "gamma": gamma, "walkers": bool(walkers)}

    def wander(self, L, m, direction, parity):
        self.lib.orc_wander(L, m, int(direction), int(parity))

    def run_ex(self, st, schedule, interval):
        """gamma daemons / walkers per spin (interval 0: the log refresh schedule)."""
        sched = np.ascontiguousarray(schedule, np.float64)
        t = ctypes.c_int64(st["t"])
        rc = self.lib.orc_run_ex(st["L"], st["S"], st["R"], st.get("gamma", 1), int(st.get("walkers", False)),
                                 st["seed"], st["J"], st["s"], st["m"], ctypes.byref(t), sched, len(sched),
                                 int(interval))
        if rc:
            raise ValueError("orc_run_ex rejected its arguments")
        st["t"] = t.value
        return st

    def run(self, st, schedule, interval, serial=False):
        sched = np.ascontiguousarray(schedule, np.float64)
        t = ctypes.c_int64(st["t"])
        rc = self.lib.orc_run(st["L"], st["S"], st["R"], st["seed"], st["J"], st["s"], st["m"],
                              ctypes.byref(t), sched, len(sched), int(interval), int(serial))
        if rc:
            raise ValueError("orc_run rejected its arguments")
        st["t"] = t.value
        return st

    def run_logrefresh(self, st, schedule):
        sched = np.ascontiguousarray(schedule, np.float64)
        t = ctypes.c_int64(st["t"])
        rc = self.lib.orc_run_logrefresh(st["L"], st["S"], st["R"], st["seed"], st["J"],
                                         st["s"], st["m"], ctypes.byref(t), sched, len(sched))
        if rc:
            raise ValueError("orc_run_logrefresh rejected its arguments")
        st["t"] = t.value
        return st

    def run_metropolis(self, st, schedule, serial=False):
        sched = np.ascontiguousarray(schedule, np.float64)
        t = ctypes.c_int64(st["t"])
        rc = self.lib.orc_run_metropolis(st["L"], st["S"], st["R"], st["seed"], st["J"],
                                         st["s"], ctypes.byref(t), sched, len(sched),
                                         int(serial))
        if rc:
            raise ValueError("orc_run_metropolis rejected its arguments")
        st["t"] = t.value
        return st

    def measure(self, st):
        S, R = st["S"], st["R"]
        e = np.zeros(S * R, np.int64)
        a = np.zeros(S * R, np.int64)
        q = np.zeros(max(1, S * R * (R - 1) // 2), np.int64)
        m = st["m"]
        gamma = st.get("gamma", 1)
        m0 = m if gamma == 1 else np.ascontiguousarray(m[:, :, 0, :])
        self.lib.orc_measure(st["L"], S, R, st["J"], st["s"], m0,
                             e.ctypes.data, a.ctypes.data, q.ctypes.data)
        if gamma > 1:  # H_aux sums every daemon of every family
            a = 4 * m.reshape(S * R, -1).astype(np.int64).sum(axis=1)
        return e, a, q[: S * R * (R - 1) // 2]

    def correlation(self, st):
        """G[S, L]: sum over pairs, axes and sites of q_x q_{x + r e_d} (Sec. 3)."""
        G = np.zeros((st["S"], st["L"]), np.int64)
        if self.lib.orc_correlation(st["L"], st["S"], st["R"], np.ascontiguousarray(st["s"], np.int8), G):
            raise ValueError("correlation needs two replicas or more")
        return G

    # -- exact enumeration ---------------------------------------------------
    def dos(self, L, J):
        N = L ** 3
        counts = np.zeros(6 * N + 1, np.int64)
        if self.lib.orc_enumerate_dos(L, np.ascontiguousarray(J, np.int8), counts):
            raise ValueError("lattice too large to enumerate")
        return counts

    def all_energies(self, L, J):
        E = np.zeros(2 ** (L ** 3), np.int64)
        if self.lib.orc_all_energies(L, np.ascontiguousarray(J, np.int8), E):
            raise ValueError("lattice too large to enumerate")
        return E

    def l2_transition_micsa(self, J, pm):
        P = np.zeros((256, 256), np.float64)
        self.lib.orc_l2_transition_micsa(np.ascontiguousarray(J, np.int8),
                                         np.ascontiguousarray(pm, np.float64), P)
        return P

    def l2_transition_metro(self, J, T):
        P = np.zeros((256, 256), np.float64)
        if self.lib.orc_l2_transition_metro(np.ascontiguousarray(J, np.int8), float(T), P):
            raise ValueError("bad temperature")
        return P
