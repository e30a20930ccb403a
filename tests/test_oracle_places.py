"""Pins of the oracle's finishing-order rollouts and place counts.

Section 3 runs a race until its last competitor crosses the line and lets betting stop
earlier (for instance when the third-placed competitor crosses); place markets need the
order of the first `places` finishers.  The pins: closed forms of noise-free races,
hand-worked within-step orders, exhaustive enumeration of tiny two-point races (an
independent implementation of the same readings in tests/exact_race.py), and invariants
(each place is taken once per rollout, the first place is the win count).
"""
from fractions import Fraction

import numpy as np
import pytest

from tests.exact_race import exact_place_probs
from tests.test_oracle_race import ENUM_CASES, race


def test_zero_noise_order_is_sorted_crossing_time(oracle_lib):
    # sigma = 0, rho = 1/2, P = 1, theta = 0: competitor c moves mu_c per step and crosses at
    # real time (L - d0_c) / mu_c, so the finishing order is the ascending order of those times
    rng = np.random.default_rng(5)
    done = 0
    while done < 30:
        n = int(rng.integers(2, 9))
        L = 1000
        d0 = rng.integers(0, 900, n)
        mu = rng.integers(3, 30, n)
        times = [Fraction(int(L - a), int(m)) for a, m in zip(d0, mu)]
        srt = sorted(times)
        if min(b - a for a, b in zip(srt, srt[1:])) < Fraction(1, 100):
            continue
        order = sorted(range(n), key=lambda c: times[c])
        r = race(d0.astype(float), mu.astype(float), theta=[0.0] * n, L=float(L))
        places = int(rng.integers(1, n + 1))
        counts, steps, st = oracle_lib.race_places(r, 0, places, R=3)
        want = np.zeros((n, places), np.int32)
        for j in range(places):
            want[order[j], j] = 3
        assert st == 0 and np.array_equal(counts, want), (d0, mu, counts)
        assert steps == 3 * int(np.ceil(float(srt[places - 1])))
        done += 1


def test_same_step_finishers_ordered_by_crossing_time_not_distance(oracle_lib):
    # A (d 5, mu 10) ends the step at 15 with tau = 0.5; B (d 9.9375, mu 0.25) ends at 10.1875
    # with tau = 0.25: B crossed first although A is farther past the line
    r = race([5.0, 9.9375], [10.0, 0.25], theta=[0.0, 0.0], L=10.0)
    order, steps, st = oracle_lib.rollout_order(r, 0, 0, 0, 2)
    assert st == 0 and steps == 1 and list(order) == [1, 0]


def test_equal_crossing_times_take_lower_index_first(oracle_lib):
    # both at 8 after two steps of 4, both cross in step 3 with tau = 0.5
    r = race([0.0, 0.0, 1.0], [4.0, 4.0, 1.0], theta=[0.0] * 3, L=10.0)
    order, steps, st = oracle_lib.rollout_order(r, 0, 0, 0, 2)
    assert st == 0 and steps == 3 and list(order) == [0, 1]
    r2 = race([0.0, 0.0, 1.0], [4.0, 4.0, 1.0], theta=[0.0] * 3, L=10.0)
    r2["d0"] = r2["d0"][[1, 0, 2]]
    order2, _, _ = oracle_lib.rollout_order(r2, 0, 0, 0, 2)
    assert list(order2) == [0, 1]


def test_finished_competitors_keep_moving_and_blocking(oracle_lib):
    # A (0.5, mu 12) crosses in the first step and keeps moving 12 per step; B (0, previous
    # step 1) trails it within theta = 100 for ten steps (the gap is 0.5 + 11 t), so it is
    # blocked and moves min(prev_B, prev_A) = 1 per step: it crosses in step 10.  If finished
    # competitors stopped moving or blocking, B would move mu_B = 5 from step 2 on.
    r = race([0.5, 0.0], [12.0, 5.0], theta=[0.0, 100.0], L=10.0, prev0=[12.0, 1.0])
    order, steps, st = oracle_lib.rollout_order(r, 0, 0, 0, 2)
    assert st == 0 and list(order) == [0, 1] and steps == 10


@pytest.mark.parametrize("case", range(len(ENUM_CASES)))
def test_two_point_places_match_exhaustive_enumeration(oracle_lib, case):
    L, d0, mu, sigma, P, theta = ENUM_CASES[case]
    n = len(d0)
    exact = exact_place_probs(L, d0, mu, sigma, n, P=P, theta=theta)
    assert np.allclose(exact.sum(0), 1.0) and np.allclose(exact.sum(1), 1.0)
    R = 100000
    r = race(d0, mu, sigma, P=P, theta=theta, L=L, dist=2, R=R, race_id=case)
    counts, steps, st = oracle_lib.race_places(r, 13, n)
    assert st == 0
    p = counts / R
    tol = 5 * np.sqrt(exact * (1 - exact) / R) + 1e-9
    assert np.all(np.abs(p - exact) <= tol), (p, exact)


def test_place_columns_sum_to_rollouts_and_first_place_is_the_win(oracle_lib):
    from paper_2108_02419_gb300 import workloads as W

    b = W.uneven_batch(seed=9, n_races=6, n_lo=2, n_hi=9, rollouts=400)
    for r in range(b.n_races):
        rc = b.race(r)
        wins, wsteps, _ = oracle_lib.race_counts(rc, b.seed)
        for places in (1, 3, rc["n"]):
            counts, steps, st = oracle_lib.race_places(rc, b.seed, places)
            k = min(places, rc["n"])
            assert st == 0
            assert np.array_equal(counts[:, 0], wins)
            assert np.all(counts[:, :k].sum(0) == 400) and np.all(counts[:, k:] == 0)
            assert np.all(counts.sum(1) <= 400)
            if places == 1:
                assert steps == wsteps
            if places >= rc["n"]:
                assert np.all(counts.sum(1) == 400)
