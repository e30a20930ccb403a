"""Pins of the oracle's finishing-order tallies (Section 3: the dry-runs estimate the outcome
distribution; the ordered top places are the outcome a forecast market is about): the noise-free
order, exhaustive enumeration of two-point races, and consistency with the pinned place counts."""
from fractions import Fraction

import numpy as np
import pytest

from tests.exact_race import exact_order_probs
from tests.test_oracle_race import ENUM_CASES, race


def decode(code, n, kk):
    out = []
    for _ in range(kk):
        out.append(code % n)
        code //= n
    return tuple(reversed(out))


def test_zero_noise_order_is_one_tuple(oracle_lib):
    # sigma = 0, rho = 1/2, P = 1, theta = 0: the order is the ascending order of the crossing
    # times (L - d0_c) / mu_c, so every rollout lands on the same tuple
    rng = np.random.default_rng(8)
    done = 0
    while done < 20:
        n = int(rng.integers(2, 8))
        L = 1000
        d0 = rng.integers(0, 900, n)
        mu = rng.integers(3, 30, n)
        times = [Fraction(int(L - a), int(m)) for a, m in zip(d0, mu)]
        srt = sorted(times)
        if min(b - a for a, b in zip(srt, srt[1:])) < Fraction(1, 100):
            continue
        order = sorted(range(n), key=lambda c: times[c])
        r = race(d0.astype(float), mu.astype(float), theta=[0.0] * n, L=float(L))
        places = int(rng.integers(1, 4))
        counts, steps, st = oracle_lib.race_orders(r, 0, places, R=5)
        kk = min(places, n)
        want = np.zeros(n ** kk, np.int32)
        code = 0
        for c in order[:kk]:
            code = code * n + c
        want[code] = 5
        assert st == 0 and np.array_equal(counts, want)
        done += 1


@pytest.mark.parametrize("case", range(len(ENUM_CASES)))
def test_two_point_orders_match_exhaustive_enumeration(oracle_lib, case):
    L, d0, mu, sigma, P, theta = ENUM_CASES[case]
    n = len(d0)
    R = 100000
    r = race(d0, mu, sigma, P=P, theta=theta, L=L, dist=2, R=R, race_id=case)
    for places in (2, 3):
        kk = min(places, n)
        exact = exact_order_probs(L, d0, mu, sigma, places, P=P, theta=theta)
        assert abs(sum(exact.values()) - 1.0) < 1e-12
        counts, steps, st = oracle_lib.race_orders(r, 17, places)
        assert st == 0 and counts.sum() == R
        for code in range(n ** kk):
            tup = decode(code, n, kk)
            q = exact.get(tup, 0.0)
            p = counts[code] / R
            assert abs(p - q) <= 5 * np.sqrt(q * (1 - q) / R) + 1e-9, (tup, p, q)


def test_marginals_are_the_place_counts(oracle_lib):
    from paper_2108_02419_gb300 import workloads as W

    b = W.uneven_batch(seed=12, n_races=6, n_lo=1, n_hi=9, rollouts=300)
    for r in range(b.n_races):
        rc = b.race(r)
        n = rc["n"]
        for places in (1, 2, 3):
            kk = min(places, n)
            orders, osteps, st = oracle_lib.race_orders(rc, b.seed, places)
            pc, psteps, st2 = oracle_lib.race_places(rc, b.seed, places)
            assert st == st2 == 0 and osteps == psteps
            table = orders.reshape((n,) * kk)
            for j in range(kk):
                axes = tuple(a for a in range(kk) if a != j)
                assert np.array_equal(table.sum(axis=axes) if axes else table, pc[:, j])
            if places == 1:
                wins, _, _ = oracle_lib.race_counts(rc, b.seed)
                assert np.array_equal(orders, wins)
