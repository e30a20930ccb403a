"""Pins of the oracle's finishing-order distribution (Section 3: the dry-runs estimate the
distribution of outcomes, and a race's full outcome is the order of all its finishers).  The
histogram of the per-rollout orders must match exhaustive enumeration of tiny two-point races
over all n! orders, collapse to the single sorted order of a noise-free race, and agree with the
pinned dense tallies and place counts."""
from fractions import Fraction

import numpy as np
import pytest

from tests.exact_race import exact_order_probs
from tests.test_oracle_race import ENUM_CASES, race


@pytest.mark.parametrize("case", range(len(ENUM_CASES)))
def test_full_orders_match_exhaustive_enumeration(oracle_lib, case):
    L, d0, mu, sigma, P, theta = ENUM_CASES[case]
    n = len(d0)
    R = 100000
    r = race(d0, mu, sigma, P=P, theta=theta, L=L, dist=2, R=R, race_id=case)
    exact = exact_order_probs(L, d0, mu, sigma, n, P=P, theta=theta)
    assert abs(sum(exact.values()) - 1.0) < 1e-12
    hist, steps, st = oracle_lib.race_order_histogram(r, 23, n)
    assert st == 0 and sum(hist.values()) == R
    assert set(hist) <= set(exact)
    for tup, q in exact.items():
        p = hist.get(tup, 0) / R
        assert abs(p - q) <= 5 * np.sqrt(q * (1 - q) / R) + 1e-9, (tup, p, q)


def test_zero_noise_full_order_is_one_permutation(oracle_lib):
    # sigma = 0, rho = 1/2, P = 1, theta = 0: every rollout finishes in the ascending order of
    # the crossing times (L - d0_c) / mu_c
    rng = np.random.default_rng(21)
    done = 0
    while done < 12:
        n = int(rng.integers(2, 10))
        L = 1000
        d0 = rng.integers(0, 900, n)
        mu = rng.integers(3, 30, n)
        times = [Fraction(int(L - a), int(m)) for a, m in zip(d0, mu)]
        srt = sorted(times)
        if min(b - a for a, b in zip(srt, srt[1:])) < Fraction(1, 100):
            continue
        order = tuple(sorted(range(n), key=lambda c: times[c]))
        r = race(d0.astype(float), mu.astype(float), theta=[0.0] * n, L=float(L))
        for places in (n, max(1, n - 2)):
            hist, _, st = oracle_lib.race_order_histogram(r, 0, places, R=7)
            assert st == 0 and dict(hist) == {order[:min(places, n)]: 7}
        done += 1


def test_agrees_with_dense_tallies_and_place_counts(oracle_lib):
    from paper_2108_02419_gb300 import workloads as W

    b = W.uneven_batch(seed=14, n_races=5, n_lo=1, n_hi=8, rollouts=400)
    for r in range(b.n_races):
        rc = b.race(r)
        n = rc["n"]
        for places in (1, 2, 3):
            kk = min(places, n)
            hist, hsteps, st = oracle_lib.race_order_histogram(rc, b.seed, places)
            dense, dsteps, st2 = oracle_lib.race_orders(rc, b.seed, places)
            assert st == st2 == 0 and hsteps == dsteps
            want = np.zeros(n ** kk, np.int64)
            for tup, c in hist.items():
                code = 0
                for o in tup:
                    code = code * n + o
                want[code] += c
            assert np.array_equal(want, dense)
        hist, _, st = oracle_lib.race_order_histogram(rc, b.seed, n)
        pc, _, _ = oracle_lib.race_places(rc, b.seed, n)
        marg = np.zeros((n, n), np.int64)
        for tup, c in hist.items():
            assert sorted(tup) == list(range(n))  # a full order is a permutation
            for j, o in enumerate(tup):
                marg[o, j] += c
        assert np.array_equal(marg, pc)


def test_cut_off_rollouts_count_for_nobody(oracle_lib):
    r = race([0.0, 0.0, 0.0], [1.0, 1.0, 1.0], sigma=[0.1, 0.1, 0.1], L=1000.0, R=5)
    hist, steps, st = oracle_lib.race_order_histogram(r, 0, 3, max_steps=10)
    assert st != 0 and sum(hist.values()) == 0 and steps == 5 * 10
