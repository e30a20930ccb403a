"""Seeded synthetic race-state generators.

This module only draws inputs: it holds none of the race simulator's arithmetic, so both
the CUDA path and the CPU oracle may take their inputs from it.  All draws use numpy's
PCG64 generator (``numpy.random.default_rng(seed)``) in float64 and are rounded once to
binary32.

Section 3 of the paper describes a race state as the positions d_c(t) of n_r competitors
on a track of length L_r plus each competitor's step-distribution parameters; the
workloads below follow the shapes of the paper's experiments (a 5-competitor race over
2000 units; batches of many independent races, Section 6).

A batch is stored as CSR over competitors: ``race_off[r] .. race_off[r+1]`` are the
competitors of race r.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DIST_NORMAL = 0
DIST_UNIFORM = 1
DIST_TWO_POINT = 2

THETA_DEFAULT = 1.0


@dataclass
class RaceBatch:
    race_off: np.ndarray  # int32 [n_races + 1]
    L: np.ndarray  # float32 [n_races]
    rollouts: np.ndarray  # int64 [n_races]
    d0: np.ndarray  # float32 [sum n]
    mu: np.ndarray
    sigma: np.ndarray
    rho: np.ndarray
    P: np.ndarray
    theta: np.ndarray
    prev0: np.ndarray | None = None  # float32 [sum n] or None (then mu * P)
    seed: int = 0
    dist: int = DIST_NORMAL
    race_id0: int = 0  # id of race 0 in the random stream
    name: str = "custom"
    meta: dict = field(default_factory=dict)
    # the time law of responsiveness (both per race, float32), or None for the position law:
    # steps elapsed before the state, and the race's expected duration in steps
    elapsed: np.ndarray | None = None
    horizon: np.ndarray | None = None

    @property
    def n_races(self) -> int:
        return int(self.race_off.shape[0] - 1)

    @property
    def n_total(self) -> int:
        return int(self.race_off[-1])

    def sizes(self) -> np.ndarray:
        return np.diff(self.race_off).astype(np.int64)

    def race(self, r: int) -> dict:
        """Per-race view (numpy slices) of race r."""
        a, b = int(self.race_off[r]), int(self.race_off[r + 1])
        out = dict(
            n=b - a,
            L=float(self.L[r]),
            d0=self.d0[a:b],
            mu=self.mu[a:b],
            sigma=self.sigma[a:b],
            rho=self.rho[a:b],
            P=self.P[a:b],
            theta=self.theta[a:b],
            prev0=None if self.prev0 is None else self.prev0[a:b],
            dist=self.dist,
            R=int(self.rollouts[r]),
            race_id=self.race_id0 + r,
        )
        if self.horizon is not None:
            out.update(law=1, t0=0.0 if self.elapsed is None else float(self.elapsed[r]), T=float(self.horizon[r]))
        return out

    def slice(self, a: int, b: int) -> "RaceBatch":
        """Races a..b-1 as a batch of their own; they keep their ids in the random stream."""
        lo, hi = int(self.race_off[a]), int(self.race_off[b])
        off = (self.race_off[a:b + 1] - lo).astype(np.int32)

        def take(x):
            return None if x is None else np.ascontiguousarray(x[lo:hi])

        per_race = lambda x: None if x is None else x[a:b].copy()
        return RaceBatch(off, self.L[a:b].copy(), self.rollouts[a:b].copy(), take(self.d0), take(self.mu),
                         take(self.sigma), take(self.rho), take(self.P), take(self.theta), take(self.prev0),
                         self.seed, self.dist, self.race_id0 + a, f"{self.name}[{a}:{b}]", dict(self.meta),
                         per_race(self.elapsed), per_race(self.horizon))


def _params(rng: np.random.Generator, n: int):
    """Per-competitor parameters: mean speed U(15,17), speed-noise std U(0.5,1.5),
    responsiveness U(0,1)."""
    mu = rng.uniform(15.0, 17.0, n).astype(np.float32)
    sigma = rng.uniform(0.5, 1.5, n).astype(np.float32)
    rho = rng.uniform(0.0, 1.0, n).astype(np.float32)
    return mu, sigma, rho


def _assemble(sizes, L, rollouts, d0, mu, sigma, rho, seed, name, dist=DIST_NORMAL, P=None, theta=None, prev0=None):
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.size + 1, dtype=np.int32)
    off[1:] = np.cumsum(sizes)
    nt = int(off[-1])
    P = np.ones(nt, np.float32) if P is None else np.asarray(P, np.float32)
    theta = np.full(nt, THETA_DEFAULT, np.float32) if theta is None else np.asarray(theta, np.float32)
    return RaceBatch(off, np.asarray(L, np.float32), np.asarray(rollouts, np.int64), np.asarray(d0, np.float32),
                     mu, sigma, rho, P, theta, prev0, seed, dist, 0, name)


def single_race_start(seed: int = 0, n: int = 5, L: float = 2000.0, rollouts: int = 1000) -> RaceBatch:
    """One race from the start line: n competitors at d = 0 on a track of length L."""
    rng = np.random.default_rng(seed)
    mu, sigma, rho = _params(rng, n)
    return _assemble([n], [L], [rollouts], np.zeros(n, np.float32), mu, sigma, rho, seed, f"single_race_n{n}_L{int(L)}_R{rollouts}")


def uniform_batch(seed: int = 0, n_races: int = 4096, n: int = 20, L: float = 5000.0, rollouts: int = 10000) -> RaceBatch:
    """Mid-race snapshots of equal size: positions U(0, 0.9 L) per competitor."""
    rng = np.random.default_rng(seed)
    nt = n_races * n
    mu, sigma, rho = _params(rng, nt)
    d0 = rng.uniform(0.0, 0.9 * L, nt).astype(np.float32)
    return _assemble(np.full(n_races, n), np.full(n_races, L), np.full(n_races, rollouts), d0, mu, sigma, rho, seed,
                     f"uniform_{n_races}x{n}_L{int(L)}_R{rollouts}")


def uneven_batch(seed: int = 0, n_races: int = 10000, n_lo: int = 2, n_hi: int = 24, L: float = 5000.0,
                 rem_lo: float = 100.0, rem_hi: float = 5000.0, r_lo_exp: float = 3.0, r_hi_exp: float = 5.0,
                 rollouts: int | None = None) -> RaceBatch:
    """Snapshots of uneven shape: competitor count uniform in [n_lo, n_hi], remaining
    distance L - d uniform in [rem_lo, rem_hi] per competitor, rollout budget
    floor(10^U(r_lo_exp, r_hi_exp)) per snapshot (or a fixed ``rollouts``)."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, n_races)
    nt = int(sizes.sum())
    mu, sigma, rho = _params(rng, nt)
    rem = rng.uniform(rem_lo, rem_hi, nt)
    d0 = (L - rem).astype(np.float32)
    if rollouts is None:
        R = np.floor(10.0 ** rng.uniform(r_lo_exp, r_hi_exp, n_races)).astype(np.int64)
    else:
        R = np.full(n_races, rollouts, np.int64)
    return _assemble(sizes, np.full(n_races, L), R, d0, mu, sigma, rho, seed,
                     f"uneven_{n_races}_n{n_lo}-{n_hi}_L{int(L)}")


def from_arrays(sizes, L, rollouts, d0, mu, sigma, rho, P=None, theta=None, prev0=None, seed=0,
                dist=DIST_NORMAL, name="custom") -> RaceBatch:
    """A batch from explicit per-race and per-competitor arrays."""
    f = lambda a: None if a is None else np.asarray(a, np.float32).ravel()
    sizes = np.atleast_1d(np.asarray(sizes, np.int64))
    L = np.broadcast_to(np.asarray(L, np.float32), sizes.shape).copy()
    rollouts = np.broadcast_to(np.asarray(rollouts, np.int64), sizes.shape).copy()
    return _assemble(sizes, L, rollouts, f(d0), f(mu), f(sigma), f(rho), seed, name, dist, f(P), f(theta), f(prev0))


def with_time_law(rb: RaceBatch, elapsed, horizon) -> RaceBatch:
    """The same batch under the time law of responsiveness: per race the steps elapsed before
    the state and the expected duration in steps (scalars broadcast)."""
    out = rb.slice(0, rb.n_races)
    out.race_id0 = rb.race_id0
    out.elapsed = np.broadcast_to(np.asarray(elapsed, np.float32), (rb.n_races,)).copy()
    out.horizon = np.broadcast_to(np.asarray(horizon, np.float32), (rb.n_races,)).copy()
    return out


def concat(batches) -> RaceBatch:
    """Concatenate batches (same seed and distribution)."""
    b0 = batches[0]
    sizes = np.concatenate([b.sizes() for b in batches])
    cat = lambda k: np.concatenate([getattr(b, k) for b in batches])
    have = [b.prev0 is not None for b in batches]
    if any(have) and not all(have):
        raise ValueError("concat: prev0 given for some batches only")
    prev0 = cat("prev0") if all(have) else None
    return _assemble(sizes, cat("L"), cat("rollouts"), cat("d0"), cat("mu"), cat("sigma"), cat("rho"), b0.seed,
                     "+".join(b.name for b in batches), b0.dist, cat("P"), cat("theta"), prev0)


def for_rank(rb: RaceBatch, rank: int) -> RaceBatch:
    """Weak scaling: rank r runs a batch of the same shape whose races take the stream ids
    r * n_races .. (r+1) * n_races - 1, so no two ranks simulate the same race."""
    out = rb.slice(0, rb.n_races)
    out.race_id0 = rb.race_id0 + rank * rb.n_races
    return out


def shard(rb: RaceBatch, rank: int, world: int) -> RaceBatch:
    """Strong scaling: a contiguous share of the races (ids kept), balanced by rollouts x competitors."""
    work = np.cumsum(rb.rollouts * rb.sizes())
    total = int(work[-1])
    bounds = [0] + [int(np.searchsorted(work, total * q / world, side="left")) + 1 for q in range(1, world)] + [rb.n_races]
    bounds = np.maximum.accumulate(np.minimum(bounds, rb.n_races))
    return rb.slice(int(bounds[rank]), int(bounds[rank + 1]))
