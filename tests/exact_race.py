"""Exact finishing distribution of tiny two-point races by exhaustive enumeration.

An independent brute-force check of the Monte Carlo estimator (Section 3: the dry-run
estimate converges to the probabilities of each outcome).  For a race whose step
generator delta(v_c) takes the two values mu_c - sigma_c and mu_c + sigma_c with
probability 1/2 each, every path of the race is enumerated and the probability mass of
each winner is summed exactly.

Restrictions that keep every operation exact, so the enumeration needs no model of
binary32 rounding except for the finish-time division: rho_c = 1/2 (so the
responsiveness R_c is exactly 1), and all positions, means, spreads, preferences and
thresholds are small dyadic rationals, so every sum, product and min is exact in both
binary32 and float64.  The within-step finish times tau_c = (L - d_c) / S_c are rounded
to binary32 like the simulator's.  Identical paths (same positions and previous steps)
are merged, so the work grows with the number of distinct states, not of paths.
"""
from __future__ import annotations

from collections import defaultdict
from itertools import product

import numpy as np

S_FLOOR = float(np.float32(1e-3))


def _nearest_in_front(d, c):
    """i+ of Section 3: the nearest competitor strictly in front of c (lowest index on ties)."""
    best = None
    for i, di in enumerate(d):
        if i == c or not di > d[c]:
            continue
        if best is None or di < d[best]:
            best = i
    return best


def exact_win_probs(L, d0, mu, sigma, P=None, theta=None, prev0=None, max_steps=200):
    n = len(d0)
    P = [1.0] * n if P is None else list(P)
    theta = [1.0] * n if theta is None else list(theta)
    prev = [mu[c] * P[c] for c in range(n)] if prev0 is None else list(prev0)
    for v in list(d0) + list(mu) + list(sigma) + P + theta + prev + [L]:
        assert float(np.float32(v)) == v and (v * 2 ** 12) == int(v * 2 ** 12), "inputs must be small dyadics"
    states = {(tuple(float(x) for x in d0), tuple(float(x) for x in prev)): 1.0}
    win = np.zeros(n)
    for _ in range(max_steps):
        nxt = defaultdict(float)
        for (d, pv), mass in states.items():
            fixed = {}
            free = []
            for c in range(n):
                ip = _nearest_in_front(d, c)
                if ip is not None and not (d[ip] - d[c] > theta[c]):
                    fixed[c] = min(pv[c], pv[ip])  # R_c = 1
                else:
                    free.append(c)
            share = mass / (2 ** len(free))
            for signs in product((-1.0, 1.0), repeat=len(free)):
                S = [0.0] * n
                for c, v in fixed.items():
                    S[c] = v
                for c, z in zip(free, signs):
                    S[c] = P[c] * (mu[c] + sigma[c] * z)
                S = [s if s >= S_FLOOR else S_FLOOR for s in S]  # Section 3: S > 0
                dn = [d[c] + S[c] for c in range(n)]
                fin = [c for c in range(n) if dn[c] >= L]
                if fin:
                    taus = [(np.float32(np.float32(L) - np.float32(d[c])) / np.float32(S[c]), c) for c in fin]
                    w = min(taus)[1]  # least tau, then lowest index
                    win[w] += share
                else:
                    nxt[(tuple(dn), tuple(S))] += share
        states = nxt
        if not states:
            break
    assert not states, "race did not end within max_steps"
    return win


def exact_order_probs(L, d0, mu, sigma, places, P=None, theta=None, prev0=None, max_steps=200):
    """Exact probability of each ordered top-kk tuple (kk = min(places, n)) of a two-point race,
    by the same enumeration: every competitor keeps moving under Eq. 1 until kk competitors have
    crossed; those crossing in one step are placed by their binary32 crossing time tau, then by
    index.  Returns {tuple of kk competitors: probability}."""
    n = len(d0)
    P = [1.0] * n if P is None else list(P)
    theta = [1.0] * n if theta is None else list(theta)
    prev = [mu[c] * P[c] for c in range(n)] if prev0 is None else list(prev0)
    for v in list(d0) + list(mu) + list(sigma) + P + theta + prev + [L]:
        assert float(np.float32(v)) == v and (v * 2 ** 12) == int(v * 2 ** 12), "inputs must be small dyadics"
    places = min(places, n)
    states = {(tuple(float(x) for x in d0), tuple(float(x) for x in prev), ()): 1.0}
    out = defaultdict(float)
    for _ in range(max_steps):
        nxt = defaultdict(float)
        for (d, pv, order), mass in states.items():
            fixed = {}
            free = []
            for c in range(n):
                ip = _nearest_in_front(d, c)
                if ip is not None and not (d[ip] - d[c] > theta[c]):
                    fixed[c] = min(pv[c], pv[ip])
                else:
                    free.append(c)
            share = mass / (2 ** len(free))
            for signs in product((-1.0, 1.0), repeat=len(free)):
                S = [0.0] * n
                for c, v in fixed.items():
                    S[c] = v
                for c, z in zip(free, signs):
                    S[c] = P[c] * (mu[c] + sigma[c] * z)
                S = [s if s >= S_FLOOR else S_FLOOR for s in S]
                dn = [d[c] + S[c] for c in range(n)]
                new = [c for c in range(n) if c not in order and dn[c] >= L]
                taus = sorted((np.float32(np.float32(L) - np.float32(d[c])) / np.float32(S[c]), c) for c in new)
                o2 = order + tuple(c for _, c in taus)
                if len(o2) >= places:
                    out[o2[:places]] += share
                else:
                    nxt[(tuple(dn), tuple(S), o2)] += share
        states = nxt
        if not states:
            break
    assert not states, "race did not end within max_steps"
    return dict(out)


def exact_place_probs(L, d0, mu, sigma, places, P=None, theta=None, prev0=None, max_steps=200):
    """Exact probability that competitor c finishes in place j (j < places) of a two-point
    race: the marginals of exact_order_probs.  Returns an [n, places] array."""
    n = len(d0)
    kk = min(places, n)
    out = np.zeros((n, kk))
    for tup, pr in exact_order_probs(L, d0, mu, sigma, places, P=P, theta=theta, prev0=prev0,
                                     max_steps=max_steps).items():
        for j, c in enumerate(tup):
            out[c, j] += pr
    return out
