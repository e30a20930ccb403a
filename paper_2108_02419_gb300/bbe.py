"""Python binding of the C ABI in include/bbe.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but
convert arguments (torch tensors, numpy arrays, raw pointers, streams) and raise
``BbeError`` on a non-zero status.  All simulation work runs in the CUDA library; there
is no fallback: if ``libbbe.so`` has not been built, importing the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BBE_LIB may name another build of the library (the checked build: build.build(checked=True))
LIB_PATH = os.environ.get("BBE_LIB") or os.path.join(_HERE, "_lib", "libbbe.so")

BBE_OK = 0
STATUS_NAMES = {0: "BBE_OK", -1: "BBE_ERR_ARG", -2: "BBE_ERR_UNSUPPORTED", -3: "BBE_ERR_FINISHED",
                -4: "BBE_ERR_CUDA", -5: "BBE_ERR_STEP_LIMIT", -6: "BBE_ERR_TIMEOUT", -7: "BBE_ERR_RANGE"}
BBE_DIST_NORMAL, BBE_DIST_UNIFORM, BBE_DIST_TWO_POINT = 0, 1, 2
BBE_MAX_COMPETITORS = 32
BBE_MAX_STEPS_DEFAULT = 1 << 20


class BbeError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        self.status = status
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {message}")


class bbe_launch_cfg(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("rollouts_per_lane", C.c_int32),
                ("max_steps", C.c_int32), ("slots_per_lane", C.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded libbbe.so.  Raises if the library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2108_02419_gb300.build.build() "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u32, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        sig = {
            "bbe_race_init": [C.POINTER(vp), i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, u64, C.c_int, u32, vp],
            "bbe_rollout_batch": [vp, vp, vp, vp],
            "bbe_win_probs": [vp, vp, vp, vp, vp],
            "bbe_place_counts": [vp, C.c_int32, vp, vp, vp],
            "bbe_order_counts": [vp, C.c_int32, vp, vp, vp, vp],
            "bbe_order_table_size": [vp, C.c_int32, C.POINTER(C.c_int64)],
            "bbe_order_histogram": [vp, i32, vp, vp, vp, vp, vp],
            "bbe_order_histogram_layout": [vp, i32, vp, vp],
            "bbe_order_key_encode": [i32, i32, vp, vp],
            "bbe_order_key_decode": [i32, i32, u64, vp],
            "bbe_race_trajectory": [vp, C.c_uint32, C.c_int32, vp, vp, vp, vp],
            "bbe_preference_coefficients": [C.c_int32, vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp],
            "bbe_snapshot_batch": [C.POINTER(vp), vp, C.c_int32, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int64, C.c_uint32, C.POINTER(C.c_int32), vp],
            "bbe_bettor_predictions": [vp, C.c_int32, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_float, C.c_uint32, vp, vp],
            "bbe_place_probs": [vp, C.c_int32, vp, C.c_int32, vp, vp],
            "bbe_batch_status": [vp, vp],
            "bbe_batch_set_cfg": [vp, C.POINTER(bbe_launch_cfg)],
            "bbe_batch_get_cfg": [vp, C.POINTER(bbe_launch_cfg)],
            "bbe_batch_autotune": [vp, vp, C.c_double, vp],
            "bbe_batch_layout": [vp, vp],
            "bbe_batch_set_law": [vp, C.c_int, vp, vp, vp],
            "bbe_batch_set_layout": [vp, vp],
            "bbe_batch_info": [vp, vp, vp, vp, vp],
            "bbe_batch_launches": [vp, vp],
            "bbe_rollout_noalloc": [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, u64, C.c_int, u32, vp, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.bbe_destroy_batch.argtypes = [vp]
        L.bbe_destroy_batch.restype = None
        L.bbe_last_error.argtypes = []
        L.bbe_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status: int, func: str):
    if status != BBE_OK:
        raise BbeError(status, func, lib().bbe_last_error().decode(errors="replace"))


def _ptr(x, dtype=None):
    """Raw address of a torch tensor / numpy array (contiguous, of the given dtype), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError(f"expected numpy {dtype}, got {x.dtype}")
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    import torch

    if isinstance(x, torch.Tensor):
        if dtype is not None and x.dtype != getattr(torch, np.dtype(dtype).name):
            raise TypeError(f"expected torch {np.dtype(dtype).name}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def bbe_race_init(n_races, race_off, track_len, rollouts, pos, mu, sigma, resp, pref=None, theta=None, prev_step=None,
                  seed=0, dist=BBE_DIST_NORMAL, race_id0=0, stream=None) -> int:
    """Stage a batch of race states; returns the opaque handle (an int)."""
    h = C.c_void_p()
    st = lib().bbe_race_init(C.byref(h), int(n_races), _ptr(race_off, np.int32), _ptr(track_len, np.float32),
                             _ptr(rollouts, np.int64), _ptr(pos, np.float32), _ptr(mu, np.float32),
                             _ptr(sigma, np.float32), _ptr(resp, np.float32), _ptr(pref, np.float32),
                             _ptr(theta, np.float32), _ptr(prev_step, np.float32), int(seed) & (2**64 - 1), int(dist),
                             int(race_id0) & 0xFFFFFFFF, _stream(stream))
    _check(st, "bbe_race_init")
    return h.value


def bbe_rollout_batch(batch: int, win_counts, steps_total=None, stream=None) -> None:
    _check(lib().bbe_rollout_batch(batch, _ptr(win_counts, np.int32), _ptr(steps_total, np.int64), _stream(stream)),
           "bbe_rollout_batch")


def bbe_win_probs(batch: int, win_counts, probs, odds=None, stream=None) -> None:
    _check(lib().bbe_win_probs(batch, _ptr(win_counts, np.int32), _ptr(probs, np.float32), _ptr(odds, np.float32),
                               _stream(stream)), "bbe_win_probs")


def bbe_place_counts(batch: int, places: int, place_counts, steps_total=None, stream=None) -> None:
    _check(lib().bbe_place_counts(batch, int(places), _ptr(place_counts, np.int32), _ptr(steps_total, np.int64),
                                  _stream(stream)), "bbe_place_counts")


def bbe_order_counts(batch: int, places: int, order_counts, place_counts=None, steps_total=None, stream=None) -> None:
    _check(lib().bbe_order_counts(batch, int(places), _ptr(order_counts, np.int32), _ptr(place_counts, np.int32),
                                  _ptr(steps_total, np.int64), _stream(stream)), "bbe_order_counts")


def bbe_order_histogram(batch: int, places: int, keys, counts, place_counts=None, steps_total=None,
                        stream=None) -> None:
    _check(lib().bbe_order_histogram(batch, int(places), _ptr(keys, np.uint64), _ptr(counts, np.int32),
                                     _ptr(place_counts, np.int32), _ptr(steps_total, np.int64), _stream(stream)),
           "bbe_order_histogram")


def bbe_order_histogram_layout(batch: int, places: int, n_races: int) -> np.ndarray:
    """Each race's first hash-table entry and the total: int64 [n_races + 1]."""
    off = np.zeros(n_races + 1, np.int64)
    _check(lib().bbe_order_histogram_layout(batch, int(places), _ptr(off), None), "bbe_order_histogram_layout")
    return off


def bbe_order_key_encode(n: int, places: int, order) -> int:
    o = np.ascontiguousarray(order, dtype=np.int32)
    out = C.c_uint64(0)
    _check(lib().bbe_order_key_encode(int(n), int(places), _ptr(o), C.byref(out)), "bbe_order_key_encode")
    return int(out.value)


def bbe_order_key_decode(n: int, places: int, key: int) -> np.ndarray:
    out = np.empty(min(int(places), int(n)), np.int32)
    _check(lib().bbe_order_key_decode(int(n), int(places), int(key), _ptr(out)), "bbe_order_key_decode")
    return out


def bbe_order_table_size(batch: int, places: int) -> int:
    out = C.c_int64()
    _check(lib().bbe_order_table_size(batch, int(places), C.byref(out)), "bbe_order_table_size")
    return out.value


def bbe_place_probs(batch: int, places: int, place_counts, top: int, probs, stream=None) -> None:
    _check(lib().bbe_place_probs(batch, int(places), _ptr(place_counts, np.int32), int(top), _ptr(probs, np.float32),
                                 _stream(stream)), "bbe_place_probs")


def bbe_preference_coefficients(n_races: int, race_off, n_competitors: int, n_factors: int, factors, preferences,
                                weights, P, stream=None) -> None:
    _check(lib().bbe_preference_coefficients(int(n_races), _ptr(race_off, np.int32), int(n_competitors),
                                             int(n_factors), _ptr(factors, np.float32), _ptr(preferences, np.float32),
                                             _ptr(weights, np.float32), _ptr(P, np.float32), _stream(stream)),
           "bbe_preference_coefficients")


def bbe_race_trajectory(batch: int, k: int, cap: int, positions, step_sizes, n_steps, stream=None) -> None:
    _check(lib().bbe_race_trajectory(batch, int(k), int(cap), _ptr(positions, np.float32),
                                     _ptr(step_sizes, np.float32), _ptr(n_steps, np.int32), _stream(stream)),
           "bbe_race_trajectory")


def bbe_snapshot_batch(src: int, race: int, positions, step_sizes, n_steps, cap: int, every: int, bettors: int,
                       dry_runs: int, race_id0: int, stream=None):
    """Returns (batch handle, number of snapshots)."""
    h = C.c_void_p()
    ns = C.c_int32(0)
    _check(lib().bbe_snapshot_batch(C.byref(h), src, int(race), _ptr(positions, np.float32),
                                    _ptr(step_sizes, np.float32), _ptr(n_steps, np.int32), int(cap), int(every),
                                    int(bettors), int(dry_runs), int(race_id0) & 0xFFFFFFFF, C.byref(ns),
                                    _stream(stream)), "bbe_snapshot_batch")
    return h.value, int(ns.value)


def bbe_bettor_predictions(src: int, race: int, positions, step_sizes, n_steps, cap: int, every: int,
                           n_snapshots: int, linex_window: int, ud_gap: float, zi_stream: int, predictions,
                           stream=None) -> None:
    _check(lib().bbe_bettor_predictions(src, int(race), _ptr(positions, np.float32), _ptr(step_sizes, np.float32),
                                        _ptr(n_steps, np.int32), int(cap), int(every), int(n_snapshots),
                                        int(linex_window), float(ud_gap), int(zi_stream) & 0xFFFFFFFF,
                                        _ptr(predictions, np.int32), _stream(stream)), "bbe_bettor_predictions")


def bbe_batch_status(batch: int, stream=None) -> None:
    _check(lib().bbe_batch_status(batch, _stream(stream)), "bbe_batch_status")


def bbe_batch_set_cfg(batch: int, warps_per_block=0, blocks_per_sm=0, rollouts_per_lane=0, max_steps=0,
                      slots_per_lane=0) -> None:
    cfg = bbe_launch_cfg(warps_per_block, blocks_per_sm, rollouts_per_lane, max_steps, slots_per_lane)
    _check(lib().bbe_batch_set_cfg(batch, C.byref(cfg)), "bbe_batch_set_cfg")


def bbe_batch_get_cfg(batch: int) -> dict:
    cfg = bbe_launch_cfg()
    _check(lib().bbe_batch_get_cfg(batch, C.byref(cfg)), "bbe_batch_get_cfg")
    return cfg.as_dict()


def bbe_batch_autotune(batch: int, win_counts, budget_ms: float = 2000.0, stream=None) -> dict:
    _check(lib().bbe_batch_autotune(batch, _ptr(win_counts, np.int32), float(budget_ms), _stream(stream)),
           "bbe_batch_autotune")
    return bbe_batch_get_cfg(batch)


LAW_POSITION, LAW_TIME = 0, 1


def bbe_batch_set_law(batch: int, law: int, elapsed=None, horizon=None, stream=None) -> None:
    _check(lib().bbe_batch_set_law(batch, int(law), _ptr(elapsed, np.float32), _ptr(horizon, np.float32),
                                   _stream(stream)), "bbe_batch_set_law")


def bbe_batch_layout(batch: int) -> np.ndarray:
    out = np.zeros(BBE_MAX_COMPETITORS + 1, np.int32)
    _check(lib().bbe_batch_layout(batch, out.ctypes.data), "bbe_batch_layout")
    return out


def bbe_batch_set_layout(batch: int, slots_by_n=None) -> None:
    tab = None if slots_by_n is None else np.ascontiguousarray(slots_by_n, np.int32)
    if tab is not None and tab.shape != (BBE_MAX_COMPETITORS + 1,):
        raise ValueError("slots_by_n must have BBE_MAX_COMPETITORS + 1 entries")
    _check(lib().bbe_batch_set_layout(batch, None if tab is None else tab.ctypes.data), "bbe_batch_set_layout")


def bbe_batch_info(batch: int) -> dict:
    nr, nc, tr, mx = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
    _check(lib().bbe_batch_info(batch, C.byref(nr), C.byref(nc), C.byref(tr), C.byref(mx)), "bbe_batch_info")
    return dict(n_races=nr.value, n_competitors=nc.value, total_rollouts=tr.value, max_competitors=mx.value)


def bbe_batch_launches(batch: int) -> int:
    k = C.c_int32()
    _check(lib().bbe_batch_launches(batch, C.byref(k)), "bbe_batch_launches")
    return k.value


def bbe_destroy_batch(batch: int) -> None:
    if batch:
        lib().bbe_destroy_batch(batch)


def bbe_rollout_noalloc(n_races, n_competitors, race_off, track_len, rollouts, pos, mu, sigma, resp, pref, theta,
                        prev_step, seed, dist, race_id0, win_counts, steps_total=None, stream=None) -> None:
    """Rollout pass that allocates no memory (device arrays only; see include/bbe.h)."""
    _check(lib().bbe_rollout_noalloc(int(n_races), int(n_competitors), _ptr(race_off, np.int32),
                                     _ptr(track_len, np.float32), _ptr(rollouts, np.int64), _ptr(pos, np.float32),
                                     _ptr(mu, np.float32), _ptr(sigma, np.float32), _ptr(resp, np.float32),
                                     _ptr(pref, np.float32), _ptr(theta, np.float32), _ptr(prev_step, np.float32),
                                     int(seed) & (2**64 - 1), int(dist), int(race_id0) & 0xFFFFFFFF,
                                     _ptr(win_counts, np.int32), _ptr(steps_total, np.int64), _stream(stream)),
           "bbe_rollout_noalloc")


def bbe_last_error() -> str:
    return lib().bbe_last_error().decode(errors="replace")


# ------------------------------------------------------------------ convenience wrapper

class Batch:
    """Owns one staged batch handle; arrays are taken from a ``workloads.RaceBatch``-like
    object (numpy, host memory: bbe_race_init copies them to the device itself)."""

    def __init__(self, rb, stream=None):
        self.rb = rb
        self.handle = bbe_race_init(rb.n_races, rb.race_off, rb.L, rb.rollouts, rb.d0, rb.mu, rb.sigma, rb.rho, rb.P,
                                    rb.theta, rb.prev0, rb.seed, rb.dist, rb.race_id0, stream)
        if getattr(rb, "horizon", None) is not None:
            el = getattr(rb, "elapsed", None)
            try:
                bbe_batch_set_law(self.handle, LAW_TIME, None if el is None else np.ascontiguousarray(el, np.float32),
                                  np.ascontiguousarray(rb.horizon, np.float32), stream)
            except BaseException:
                bbe_destroy_batch(self.handle)
                raise

    def new_outputs(self, device="cuda"):
        import torch

        counts = torch.empty(self.rb.n_total, dtype=torch.int32, device=device)
        steps = torch.empty(self.rb.n_races, dtype=torch.int64, device=device)
        return counts, steps

    def rollout(self, counts=None, steps=None, stream=None):
        if counts is None:
            counts, steps = self.new_outputs()
        bbe_rollout_batch(self.handle, counts, steps, stream)
        return counts, steps

    def win_probs(self, counts, probs=None, odds=None, stream=None):
        import torch

        if probs is None:
            probs = torch.empty(self.rb.n_total, dtype=torch.float32, device=counts.device)
            odds = torch.empty_like(probs)
        bbe_win_probs(self.handle, counts, probs, odds, stream)
        return probs, odds

    def places(self, places: int, counts=None, steps=None, stream=None):
        """Place counts [sum n, places] (device int32) and steps per race (device int64)."""
        import torch

        if counts is None:
            counts = torch.empty((self.rb.n_total, places), dtype=torch.int32, device="cuda")
            steps = torch.empty(self.rb.n_races, dtype=torch.int64, device="cuda")
        bbe_place_counts(self.handle, places, counts, steps, stream)
        return counts, steps

    def orders(self, places: int, with_places: bool = False, stream=None):
        """Order tallies (device int32, every race's n_r ** min(places, n_r) table back to back),
        optionally the place counts of the same pass, and steps per race."""
        import torch

        total = bbe_order_table_size(self.handle, places)
        counts = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
        pc = torch.empty((self.rb.n_total, places), dtype=torch.int32, device="cuda") if with_places else None
        steps = torch.empty(self.rb.n_races, dtype=torch.int64, device="cuda")
        bbe_order_counts(self.handle, places, counts, pc, steps, stream)
        return counts[:total], pc, steps

    def order_histogram(self, places: int, with_places: bool = False, stream=None):
        """Finishing-order hash tables (device uint64 keys and int32 counts; race r's table is
        entries off[r] .. off[r+1]-1, unused entries hold key 2^64 - 1 and count 0), the layout
        off (host int64), optionally the place counts of the same pass, and steps per race."""
        import torch

        off = bbe_order_histogram_layout(self.handle, places, self.rb.n_races)
        total = int(off[-1])
        keys = torch.empty(total, dtype=torch.uint64, device="cuda")
        counts = torch.empty(total, dtype=torch.int32, device="cuda")
        pc = torch.empty((self.rb.n_total, places), dtype=torch.int32, device="cuda") if with_places else None
        steps = torch.empty(self.rb.n_races, dtype=torch.int64, device="cuda")
        bbe_order_histogram(self.handle, places, keys, counts, pc, steps, stream)
        return keys, counts, off, pc, steps

    def place_probs(self, counts, top: int, probs=None, stream=None):
        import torch

        if probs is None:
            probs = torch.empty(self.rb.n_total, dtype=torch.float32, device=counts.device)
        bbe_place_probs(self.handle, counts.shape[1], counts, top, probs, stream)
        return probs

    def status(self, stream=None):
        bbe_batch_status(self.handle, stream)

    def set_cfg(self, **kw):
        bbe_batch_set_cfg(self.handle, **kw)

    def cfg(self):
        return bbe_batch_get_cfg(self.handle)

    def layout(self):
        return bbe_batch_layout(self.handle)

    def set_layout(self, slots_by_n=None):
        bbe_batch_set_layout(self.handle, slots_by_n)

    def autotune(self, counts, budget_ms=2000.0, stream=None):
        return bbe_batch_autotune(self.handle, counts, budget_ms, stream)

    def close(self):
        if self.handle:
            bbe_destroy_batch(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ surrogate (include/bbe_surrogate.h)

class bbe_train_cfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float), ("batch_states", C.c_int32), ("steps", C.c_int32),
                ("shuffle_seed", C.c_uint64)]


_sg_ready = False


def _sg():
    global _sg_ready
    L = lib()
    if not _sg_ready:
        vp = C.c_void_p
        sig = {
            "bbe_surrogate_create": [C.POINTER(vp), C.c_uint64],
            "bbe_surrogate_set_params": [vp, vp],
            "bbe_surrogate_get_params": [vp, vp],
            "bbe_surrogate_train": [vp, vp, vp, C.POINTER(bbe_train_cfg), vp, vp],
            "bbe_surrogate_grad": [vp, vp, vp, vp, vp, vp],
            "bbe_surrogate_forward": [vp, vp, vp, vp],
            "bbe_surrogate_infer": [vp, vp, vp, vp, vp],
            "bbe_surrogate_status": [vp, vp],
            "bbe_surrogate_wait_probe": [vp, C.c_int64, vp],
            "bbe_surrogate_set_inputs": [vp, C.c_int32],
            "bbe_surrogate_set_gate": [vp, C.c_float],
            "bbe_surrogate_set_fallback": [vp, C.c_int64, C.c_double],
            "bbe_surrogate_fallback_budget": [C.c_int32, vp, C.c_int64, C.c_int64, C.c_double, C.POINTER(C.c_int64)],
            "bbe_surrogate_fallback_stats": [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
            "bbe_surrogate_fallback_times": [vp, vp],
            "bbe_surrogate_save": [vp, C.c_char_p],
            "bbe_surrogate_load": [C.POINTER(vp), C.c_char_p],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.bbe_surrogate_num_params.argtypes = []
        L.bbe_surrogate_num_params.restype = C.c_int64
        L.bbe_surrogate_destroy.argtypes = [vp]
        L.bbe_surrogate_destroy.restype = None
        _sg_ready = True
    return L


def bbe_surrogate_num_params() -> int:
    return int(_sg().bbe_surrogate_num_params())


def bbe_surrogate_create(init_seed: int = 0) -> int:
    h = C.c_void_p()
    _check(_sg().bbe_surrogate_create(C.byref(h), int(init_seed) & (2**64 - 1)), "bbe_surrogate_create")
    return h.value


def bbe_surrogate_set_params(s: int, params) -> None:
    p = np.ascontiguousarray(params, np.float32)
    if p.size != bbe_surrogate_num_params():
        raise ValueError("wrong parameter count")
    _check(_sg().bbe_surrogate_set_params(s, _ptr(p)), "bbe_surrogate_set_params")


def bbe_surrogate_get_params(s: int) -> np.ndarray:
    p = np.empty(bbe_surrogate_num_params(), np.float32)
    _check(_sg().bbe_surrogate_get_params(s, _ptr(p)), "bbe_surrogate_get_params")
    return p


def bbe_surrogate_train(s: int, batch: int, target_probs, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                        weight_decay=0.0, batch_states=4096, steps=1, shuffle_seed=0, loss_log=None,
                        stream=None) -> None:
    cfg = bbe_train_cfg(lr, beta1, beta2, eps, weight_decay, batch_states, steps, shuffle_seed)
    _check(_sg().bbe_surrogate_train(s, batch, _ptr(target_probs, np.float32), C.byref(cfg),
                                     _ptr(loss_log, np.float32), _stream(stream)), "bbe_surrogate_train")


def bbe_surrogate_grad(s: int, batch: int, target_probs, grad, loss=None, stream=None) -> None:
    _check(_sg().bbe_surrogate_grad(s, batch, _ptr(target_probs, np.float32), _ptr(grad, np.float32),
                                    _ptr(loss, np.float32), _stream(stream)), "bbe_surrogate_grad")


def bbe_surrogate_forward(s: int, batch: int, probs, stream=None) -> None:
    _check(_sg().bbe_surrogate_forward(s, batch, _ptr(probs, np.float32), _stream(stream)), "bbe_surrogate_forward")


def bbe_surrogate_infer(s: int, batch: int, probs, used_mc=None, stream=None) -> None:
    _check(_sg().bbe_surrogate_infer(s, batch, _ptr(probs, np.float32), _ptr(used_mc, np.uint8), _stream(stream)),
           "bbe_surrogate_infer")


SURROGATE_INPUTS_RAW, SURROGATE_INPUTS_DERIVED = 5, 14


def bbe_surrogate_set_inputs(s: int, inputs: int) -> None:
    _check(_sg().bbe_surrogate_set_inputs(s, int(inputs)), "bbe_surrogate_set_inputs")


def bbe_surrogate_set_gate(s: int, runner_up_max: float) -> None:
    """Send races whose second-largest network probability exceeds runner_up_max to Monte Carlo."""
    _check(_sg().bbe_surrogate_set_gate(s, float(runner_up_max)), "bbe_surrogate_set_gate")


def bbe_surrogate_set_fallback(s: int, pilot_rollouts: int, max_sd: float = 0.0) -> None:
    """Two-stage Monte Carlo fallback: pilot_rollouts first, then the budget rule's total
    (pilot_rollouts = 0: each race's own budget)."""
    _check(_sg().bbe_surrogate_set_fallback(s, int(pilot_rollouts), float(max_sd)), "bbe_surrogate_set_fallback")


def bbe_surrogate_fallback_budget(counts, pilot: int, cap: int, max_sd: float) -> int:
    """The fallback's budget rule for one race's pilot win counts (host int32 array)."""
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.int32))
    out = C.c_int64()
    _check(_sg().bbe_surrogate_fallback_budget(int(c.size), c.ctypes.data_as(C.c_void_p), int(pilot), int(cap),
                                               float(max_sd), C.byref(out)), "bbe_surrogate_fallback_budget")
    return out.value


def bbe_surrogate_fallback_times(s: int) -> np.ndarray:
    out = np.zeros(5, np.float64)
    _check(_sg().bbe_surrogate_fallback_times(s, out.ctypes.data), "bbe_surrogate_fallback_times")
    return out


def bbe_surrogate_fallback_stats(s: int) -> tuple:
    """(races sent to Monte Carlo, rollouts behind their answers) of the last infer call."""
    races, rollouts = C.c_int64(), C.c_int64()
    _check(_sg().bbe_surrogate_fallback_stats(s, C.byref(races), C.byref(rollouts)), "bbe_surrogate_fallback_stats")
    return races.value, rollouts.value


def bbe_surrogate_status(s: int, stream=None) -> None:
    """Synchronise and raise BBEError(BBE_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(_sg().bbe_surrogate_status(s, _stream(stream)), "bbe_surrogate_status")


def bbe_surrogate_wait_probe(s: int, limit_ns: int, stream=None) -> None:
    """Make one bounded device wait give up (no fault); the next status call reports it."""
    _check(_sg().bbe_surrogate_wait_probe(s, int(limit_ns), _stream(stream)), "bbe_surrogate_wait_probe")


def bbe_surrogate_save(s: int, path: str) -> None:
    _check(_sg().bbe_surrogate_save(s, str(path).encode()), "bbe_surrogate_save")


def bbe_surrogate_load(path: str) -> int:
    h = C.c_void_p()
    _check(_sg().bbe_surrogate_load(C.byref(h), str(path).encode()), "bbe_surrogate_load")
    return h.value


def bbe_surrogate_destroy(s: int) -> None:
    if s:
        _sg().bbe_surrogate_destroy(s)
