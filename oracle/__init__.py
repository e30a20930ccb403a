"""CPU oracle of the BBE race simulator's Monte Carlo win-probability path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg are the only callers.  Nothing on the product path imports this package,
and it imports nothing from the product package except the seeded input generators.

The arithmetic lives in ``bbe_oracle.c`` (plain C, binary32, no fused operations except
the written ``fmaf`` calls); this module compiles it with gcc and wraps it with ctypes.
``surrogate_ref.py`` holds the float64 reference of the surrogate network.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from collections import Counter
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bbe_oracle.c")
_HDR = os.path.join(_HERE, "bbe_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libbbe_oracle.so")
_lock = threading.Lock()
_lib = None

DIST_NORMAL, DIST_UNIFORM, DIST_TWO_POINT = 0, 1, 2
MAX_STEPS_DEFAULT = 1 << 20
STEP_LIMIT = -5
LAW_POSITION, LAW_TIME = 0, 1  # responsiveness laws (bbe_oracle.c: responsiveness, responsiveness_time)

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall", "-Wextra"]


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file (this one, or a test's deliberately broken copy)."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-I", _HERE, "-o", tmp, src, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (contraction off, no fast-math). Returns the .so path.

    The environment variable BBE_ORACLE_LIB names another build to load instead (the
    mutation tests use it to run the pins against broken copies)."""
    if os.environ.get("BBE_ORACLE_LIB"):
        return os.environ["BBE_ORACLE_LIB"]
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_SO) or max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_SO)
    if stale:
        compile_source(_SRC, _SO)
    return _SO


class _Race(C.Structure):
    _fields_ = [("n", C.c_int), ("L", C.c_float), ("d0", C.c_void_p), ("mu", C.c_void_p), ("sigma", C.c_void_p),
                ("rho", C.c_void_p), ("P", C.c_void_p), ("theta", C.c_void_p), ("prev0", C.c_void_p),
                ("dist", C.c_int), ("law", C.c_int), ("t0", C.c_float), ("T", C.c_float)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, u32, u64, f32 = C.c_void_p, C.c_int64, C.c_uint32, C.c_uint64, C.c_float
            L.bbe_oracle_philox4x32_10.argtypes = [vp, vp, vp]
            L.bbe_oracle_log.argtypes = [f32]
            L.bbe_oracle_log.restype = f32
            L.bbe_oracle_z.argtypes = [C.c_int, u64, u32, u32, u32, u32]
            L.bbe_oracle_z.restype = f32
            L.bbe_oracle_rollout.argtypes = [C.POINTER(_Race), u64, u32, u32, i64, vp, vp, i64]
            L.bbe_oracle_rollout.restype = C.c_int
            L.bbe_oracle_race_counts.argtypes = [C.POINTER(_Race), u64, u32, i64, i64, i64, vp, vp]
            L.bbe_oracle_race_counts.restype = C.c_int
            L.bbe_oracle_rollout_order.argtypes = [C.POINTER(_Race), u64, u32, u32, C.c_int, i64, vp, vp]
            L.bbe_oracle_rollout_order.restype = C.c_int
            L.bbe_oracle_race_places.argtypes = [C.POINTER(_Race), u64, u32, i64, i64, C.c_int, i64, vp, vp]
            L.bbe_oracle_race_places.restype = C.c_int
            L.bbe_oracle_race_orders.argtypes = [C.POINTER(_Race), u64, u32, i64, i64, C.c_int, i64, vp, vp]
            L.bbe_oracle_race_orders.restype = C.c_int
            L.bbe_oracle_race_order_list.argtypes = [C.POINTER(_Race), u64, u32, i64, i64, C.c_int, i64, vp, vp]
            L.bbe_oracle_race_order_list.restype = C.c_int
            L.bbe_oracle_trajectory.argtypes = [C.POINTER(_Race), u64, u32, u32, i64, vp, vp, vp, i64]
            L.bbe_oracle_trajectory.restype = C.c_int
            L.bbe_oracle_preference.argtypes = [C.c_int, vp, C.c_int, vp, vp, vp, vp]
            L.bbe_oracle_win_probs.argtypes = [C.c_int, vp, i64, vp, vp]
            L.bbe_oracle_log_batch.argtypes = [vp, vp, i64]
            L.bbe_oracle_sincos2pi_batch.argtypes = [vp, vp, vp, i64]
            L.bbe_oracle_z_batch.argtypes = [C.c_int, u64, u32, u32, i64, u32, u32, vp]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().bbe_oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def log_f32(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().bbe_oracle_log_batch(_ptr(x), _ptr(y), x.size)
    return y


def sincos2pi(m24):
    m = np.ascontiguousarray(m24, np.uint32)
    s = np.empty(m.shape, np.float32)
    c = np.empty(m.shape, np.float32)
    lib().bbe_oracle_sincos2pi_batch(_ptr(m), _ptr(s), _ptr(c), m.size)
    return s, c


def z(dist: int, seed: int, r: int, k: int, t: int, c: int) -> float:
    return float(lib().bbe_oracle_z(dist, seed, r, k, t, c))


def z_block(dist: int, seed: int, r: int, k0: int, nk: int, nt: int, c: int) -> np.ndarray:
    """z for rollouts k0..k0+nk-1 and steps 0..nt-1 of competitor c of race r: [nk, nt]."""
    out = np.empty((nk, nt), np.float32)
    lib().bbe_oracle_z_batch(dist, seed, r, k0, nk, nt, c, _ptr(out))
    return out


class _RaceArgs:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, race: dict):
        f = lambda a: None if a is None else np.ascontiguousarray(a, np.float32)
        self.arrays = [f(race[k]) for k in ("d0", "mu", "sigma", "rho", "P", "theta", "prev0")]
        d0, mu, sigma, rho, P, theta, prev0 = self.arrays
        self.s = _Race(int(race["n"]), float(race["L"]), _ptr(d0), _ptr(mu), _ptr(sigma), _ptr(rho), _ptr(P),
                       _ptr(theta), _ptr(prev0), int(race.get("dist", DIST_NORMAL)), int(race.get("law", LAW_POSITION)),
                       float(race.get("t0", 0.0)), float(race.get("T", 1.0)))


def rollout(race: dict, seed: int, r: int, k: int, max_steps: int = MAX_STEPS_DEFAULT, traj_cap: int = 0):
    """One dry-run: (winner, steps, trajectory [steps, n] or None)."""
    a = _RaceArgs(race)
    steps = np.zeros(1, np.int64)
    traj = np.zeros((max(traj_cap, 0), race["n"]), np.float32) if traj_cap > 0 else None
    w = lib().bbe_oracle_rollout(C.byref(a.s), seed, r, k, max_steps, _ptr(steps), _ptr(traj), traj_cap)
    st = int(steps[0])
    return w, st, (traj[: min(st, traj_cap)] if traj is not None else None)


def race_counts(race: dict, seed: int, r: int | None = None, R: int | None = None, k_begin: int = 0,
                max_steps: int = MAX_STEPS_DEFAULT):
    """Win counts of one race over rollouts k_begin .. k_begin+R-1: (counts int32 [n], steps_total, status)."""
    a = _RaceArgs(race)
    r = race["race_id"] if r is None else r
    R = race["R"] if R is None else R
    counts = np.zeros(race["n"], np.int32)
    steps = np.zeros(1, np.int64)
    st = lib().bbe_oracle_race_counts(C.byref(a.s), seed, r, k_begin, R, max_steps, _ptr(counts), _ptr(steps))
    return counts, int(steps[0]), int(st)


def trajectory(race: dict, seed: int, r: int, k: int, max_steps: int = MAX_STEPS_DEFAULT, cap: int = 100000):
    """A full run to the last finisher: (positions [steps, n], step sizes [steps, n], steps, status)."""
    a = _RaceArgs(race)
    steps = np.zeros(1, np.int64)
    d = np.zeros((cap, race["n"]), np.float32)
    s = np.zeros((cap, race["n"]), np.float32)
    st = lib().bbe_oracle_trajectory(C.byref(a.s), seed, r, k, max_steps, _ptr(steps), _ptr(d), _ptr(s), cap)
    T = int(steps[0])
    return d[:min(T, cap)], s[:min(T, cap)], T, int(st)


def rollout_order(race: dict, seed: int, r: int, k: int, places: int, max_steps: int = MAX_STEPS_DEFAULT):
    """One dry-run to the places-th finisher: (order int32 [places], steps, status)."""
    a = _RaceArgs(race)
    steps = np.zeros(1, np.int64)
    order = np.full(race["n"], -1, np.int32)
    st = lib().bbe_oracle_rollout_order(C.byref(a.s), seed, r, k, places, max_steps, _ptr(steps), _ptr(order))
    return order[:places], int(steps[0]), int(st)


def race_places(race: dict, seed: int, places: int, r: int | None = None, R: int | None = None, k_begin: int = 0,
                max_steps: int = MAX_STEPS_DEFAULT):
    """Place counts of one race: (counts int32 [n, places], steps_total, status)."""
    a = _RaceArgs(race)
    r = race["race_id"] if r is None else r
    R = race["R"] if R is None else R
    counts = np.zeros((race["n"], places), np.int32)
    steps = np.zeros(1, np.int64)
    st = lib().bbe_oracle_race_places(C.byref(a.s), seed, r, k_begin, R, places, max_steps, _ptr(counts), _ptr(steps))
    return counts, int(steps[0]), int(st)


def race_orders(race: dict, seed: int, places: int, r: int | None = None, R: int | None = None, k_begin: int = 0,
                max_steps: int = MAX_STEPS_DEFAULT):
    """Ordered top-kk tallies of one race, kk = min(places, n): (counts int32 [n ** kk], entry
    ((o_1 n + o_2) n + ..) + o_kk, steps_total, status)."""
    a = _RaceArgs(race)
    r = race["race_id"] if r is None else r
    R = race["R"] if R is None else R
    kk = min(places, race["n"])
    counts = np.zeros(race["n"] ** kk, np.int32)
    steps = np.zeros(1, np.int64)
    st = lib().bbe_oracle_race_orders(C.byref(a.s), seed, r, k_begin, R, places, max_steps, _ptr(counts), _ptr(steps))
    return counts, int(steps[0]), int(st)


def race_order_histogram(race: dict, seed: int, places: int, r: int | None = None, R: int | None = None,
                         k_begin: int = 0, max_steps: int = MAX_STEPS_DEFAULT):
    """Distribution of finishing orders of one race (Section 3): a Counter from each ordered
    tuple of the first kk = min(places, n) finishers to the number of rollouts that ended in it
    (cut-off rollouts count for nobody), the steps total and the status."""
    a = _RaceArgs(race)
    r = race["race_id"] if r is None else r
    R = race["R"] if R is None else R
    kk = min(places, race["n"])
    orders = np.empty((R, kk), np.int32)
    steps = np.zeros(1, np.int64)
    st = lib().bbe_oracle_race_order_list(C.byref(a.s), seed, r, k_begin, R, places, max_steps, _ptr(orders),
                                          _ptr(steps))
    hist = Counter(tuple(int(c) for c in row) for row in orders if row[0] >= 0)
    return hist, int(steps[0]), int(st)


def batch_order_histograms(batch, places: int, races=None, threads: int | None = None,
                           max_steps: int = MAX_STEPS_DEFAULT):
    """race_order_histogram for the given races of a RaceBatch (a thread pool over races):
    (list of Counters in the order given, steps int64 [len(races)], status)."""
    races = list(range(batch.n_races)) if races is None else [int(x) for x in races]
    threads = threads or os.cpu_count() or 1

    def one(r):
        return race_order_histogram(batch.race(r), batch.seed, places, max_steps=max_steps)

    if threads <= 1 or len(races) <= 1:
        res = [one(r) for r in races]
    else:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, races))
    status = next((st for _, _, st in res if st != 0), 0)
    return [h for h, _, _ in res], np.array([s for _, s, _ in res], np.int64), status


def batch_orders(batch, places: int, races=None, threads: int | None = None, max_steps: int = MAX_STEPS_DEFAULT,
                 rollout_chunk: int = 2500):
    """Order tallies for the given races of a RaceBatch: (list of int32 [n_r ** kk_r] arrays in
    the order given, steps int64 [len(races)], status); rollout chunks run on a thread pool."""
    races = list(range(batch.n_races)) if races is None else [int(x) for x in races]
    threads = threads or os.cpu_count() or 1
    tasks = []
    for i, r in enumerate(races):
        R = int(batch.rollouts[r])
        for k0 in range(0, R, rollout_chunk):
            tasks.append((i, r, k0, min(rollout_chunk, R - k0)))

    def one(task):
        i, r, k0, cnt = task
        return race_orders(batch.race(r), batch.seed, places, R=cnt, k_begin=k0, max_steps=max_steps)

    if threads <= 1 or len(tasks) <= 1:
        res = [one(t) for t in tasks]
    else:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, tasks))
    per_race = []
    for r in races:
        n = int(batch.race_off[r + 1] - batch.race_off[r])
        per_race.append(np.zeros(n ** min(places, n), np.int64))
    steps = np.zeros(len(races), np.int64)
    status = 0
    for (i, r, k0, cnt), (c, st, s) in zip(tasks, res):
        per_race[i] += c
        steps[i] += st
        status = min(status, s)
    return [c.astype(np.int32) for c in per_race], steps, status


def batch_places(batch, places: int, races=None, threads: int | None = None, max_steps: int = MAX_STEPS_DEFAULT,
                 rollout_chunk: int = 2500):
    """Place counts for the given races of a RaceBatch: (counts int32 [sum n, places] in the
    order given, steps int64 [len(races)], status); rollout chunks run on a thread pool."""
    races = list(range(batch.n_races)) if races is None else [int(x) for x in races]
    threads = threads or os.cpu_count() or 1
    tasks = []
    for i, r in enumerate(races):
        R = int(batch.rollouts[r])
        for k0 in range(0, R, rollout_chunk):
            tasks.append((i, r, k0, min(rollout_chunk, R - k0)))

    def one(task):
        i, r, k0, cnt = task
        return race_places(batch.race(r), batch.seed, places, R=cnt, k_begin=k0, max_steps=max_steps)

    if threads <= 1 or len(tasks) <= 1:
        res = [one(t) for t in tasks]
    else:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, tasks))
    per_race = [np.zeros((int(batch.race_off[r + 1] - batch.race_off[r]), places), np.int64) for r in races]
    steps = np.zeros(len(races), np.int64)
    status = 0
    for (i, r, k0, cnt), (c, st, s) in zip(tasks, res):
        per_race[i] += c
        steps[i] += st
        status = min(status, s)
    counts = np.concatenate(per_race).astype(np.int32) if per_race else np.zeros((0, places), np.int32)
    return counts, steps, status


def batch_counts(batch, races=None, threads: int | None = None, max_steps: int = MAX_STEPS_DEFAULT,
                 rollout_chunk: int = 2500):
    """Win counts for the given races of a RaceBatch (all by default).  Each race's rollouts
    are split into chunks of ``rollout_chunk`` and the chunks run on a thread pool (ctypes
    releases the GIL); the counter-based stream makes the split exact.  Returns
    (counts int32 [sum n over the given races, concatenated in the order given],
    steps int64 [len(races)], status)."""
    races = list(range(batch.n_races)) if races is None else [int(x) for x in races]
    threads = threads or os.cpu_count() or 1
    tasks = []
    for i, r in enumerate(races):
        R = int(batch.rollouts[r])
        for k0 in range(0, R, rollout_chunk):
            tasks.append((i, r, k0, min(rollout_chunk, R - k0)))

    def one(task):
        i, r, k0, cnt = task
        return race_counts(batch.race(r), batch.seed, R=cnt, k_begin=k0, max_steps=max_steps)

    if threads <= 1 or len(tasks) <= 1:
        res = [one(t) for t in tasks]
    else:
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(one, tasks))
    per_race = [np.zeros(int(batch.race_off[r + 1] - batch.race_off[r]), np.int64) for r in races]
    steps = np.zeros(len(races), np.int64)
    status = 0
    for (i, r, k0, cnt), (c, st, s) in zip(tasks, res):
        per_race[i] += c
        steps[i] += st
        status = min(status, s)
    counts = np.concatenate(per_race).astype(np.int32) if per_race else np.zeros(0, np.int32)
    return counts, steps, status


def preference(race_off, factors, prefs, weights) -> np.ndarray:
    """P per competitor from factor vectors [n_races, F], preference vectors [sum n, F] and weights [F]."""
    off = np.ascontiguousarray(race_off, np.int32)
    f = np.ascontiguousarray(factors, np.float32)
    p = np.ascontiguousarray(prefs, np.float32)
    w = np.ascontiguousarray(weights, np.float32)
    F = w.size
    assert f.shape == (off.size - 1, F) and p.shape == (int(off[-1]), F)
    out = np.empty(int(off[-1]), np.float32)
    lib().bbe_oracle_preference(off.size - 1, _ptr(off), F, _ptr(f), _ptr(p), _ptr(w), _ptr(out))
    return out


def win_probs(counts, R: int):
    counts = np.ascontiguousarray(counts, np.int32)
    p = np.empty(counts.size, np.float32)
    o = np.empty(counts.size, np.float32)
    lib().bbe_oracle_win_probs(counts.size, _ptr(counts), R, _ptr(p), _ptr(o))
    return p, o
