"""Pins of the oracle's race simulator (Section 3, Eq. 1) and dry-run estimator.

Each test fixes a case whose answer follows from the paper's definitions or from
mathematics without running the oracle's own formulas: hand-worked steps, closed forms
for noise-free races, exhaustive enumeration of tiny two-point races, and invariants of
the estimator (counts sum to R, symmetry, monotonicity).
"""
from fractions import Fraction

import numpy as np
import pytest

from tests.exact_race import exact_win_probs


def race(d0, mu, sigma=None, rho=None, P=None, theta=None, prev0=None, L=100.0, dist=0, R=1, race_id=0):
    n = len(d0)
    f = lambda v, default: np.asarray([default] * n if v is None else v, np.float32)
    return dict(n=n, L=float(L), d0=f(d0, 0), mu=f(mu, 0), sigma=f(sigma, 0.0), rho=f(rho, 0.5), P=f(P, 1.0),
                theta=f(theta, 1.0), prev0=None if prev0 is None else f(prev0, 0), dist=dist, R=R, race_id=race_id)


def steps_of(traj, d0):
    full = np.vstack([np.asarray(d0, np.float32)[None, :], traj])
    return np.diff(full, axis=0)


# ------------------------------------------------------------------ hand-worked steps

def test_constant_speed_single_competitor(oracle_lib):
    # sigma = 0, rho = 1/2 (R = 1), P = 1: the step is exactly mu; 16 * 125 = 2000 = L
    w, steps, traj = oracle_lib.rollout(race([0.0], [16.0], L=2000.0), 0, 0, 0, traj_cap=200)
    assert w == 0 and steps == 125
    assert np.array_equal(traj[:, 0], 16.0 * np.arange(1, 126, dtype=np.float32))


def test_preference_scales_the_step(oracle_lib):
    # Eq. 1 first case: S = R P delta; P = 1/2 halves every step
    w, steps, traj = oracle_lib.rollout(race([0.0], [16.0], P=[0.5], L=2000.0), 0, 0, 0, traj_cap=300)
    assert steps == 250 and np.all(steps_of(traj, [0.0]) == 8.0)


def test_step_floor_keeps_steps_positive(oracle_lib):
    # Section 3 requires S > 0; a vanishing mean step is floored at 1e-3
    w, steps, traj = oracle_lib.rollout(race([0.0], [1e-6], L=0.01), 0, 0, 0, traj_cap=20)
    d, want = np.float32(0.0), []
    while not want or want[-1] < np.float32(0.01):
        d = np.float32(d + np.float32(1e-3))  # binary32 position update
        want.append(d)
    assert steps == len(want) and np.array_equal(traj[:, 0], np.array(want, np.float32))


@pytest.mark.parametrize("rho,direction", [(1.0, +1), (0.0, -1), (0.75, +1), (0.25, -1)])
def test_responsiveness_fades_or_finishes(oracle_lib, rho, direction):
    # R_c lets a competitor start slow and finish fast (rho > 1/2) or start fast and fade
    # (rho < 1/2): with sigma = 0 the steps change monotonically along the track, are mu at
    # mid-track and stay within mu (1 -+ kappa |2 rho - 1| / 2), kappa = 0.2
    mu, L = 10.0, 1000.0
    w, steps, traj = oracle_lib.rollout(race([0.0], [mu], rho=[rho], L=L), 0, 0, 0, traj_cap=200)
    s = steps_of(traj, [0.0])[:, 0].astype(np.float64)
    d_before = np.concatenate([[0.0], traj[:-1, 0]]).astype(np.float64)
    assert np.all(direction * np.diff(s) > 0)
    amp = 0.2 * abs(2 * rho - 1) / 2
    assert abs(s[0] - mu * (1 - direction * amp)) < 1e-5 * mu
    frac = d_before / L
    expect = mu * (1 + direction * 0.2 * abs(2 * rho - 1) * (frac - 0.5))
    assert np.max(np.abs(s - expect)) < 1e-5 * mu  # linear law, to binary32 rounding


def test_blocked_competitor_follows_slower_leader(oracle_lib):
    # c0 (mu 10) starts 0.5 behind c1 (mu 4), theta 1: Delta = 0.5 <= theta, so c0 is
    # blocked and its step is min(S_c0(t-1), S_c1(t-1)) = 4 (Eq. 1, delta_min); the gap
    # never grows past theta and the slower c1 always wins.
    r = race([0.0, 0.5], [10.0, 4.0], L=100.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=100)
    assert np.all(steps_of(traj, [0.0, 0.5]) == 4.0)
    assert w == 1
    counts, _, st = oracle_lib.race_counts(r, 0, R=50)
    assert st == 0 and list(counts) == [0, 50]


def test_unblocked_when_gap_exceeds_threshold(oracle_lib):
    # same race with theta_c0 = 0.25 < Delta: c0 runs free at 10 and wins every time
    r = race([0.0, 0.5], [10.0, 4.0], theta=[0.25, 1.0], L=100.0)
    counts, _, _ = oracle_lib.race_counts(r, 0, R=50)
    assert list(counts) == [50, 0]


def test_gap_equal_to_threshold_blocks(oracle_lib):
    # Eq. 1: the free branch needs Delta > theta strictly
    r = race([0.0, 0.5], [10.0, 4.0], theta=[0.5, 1.0], L=100.0)
    counts, _, _ = oracle_lib.race_counts(r, 0, R=20)
    assert list(counts) == [0, 20]


def test_delta_min_uses_slower_of_the_two(oracle_lib):
    # a blocked competitor that is itself slower keeps its own previous step
    r = race([0.0, 0.5], [3.0, 4.0], L=100.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=3)
    s = steps_of(traj, [0.0, 0.5])
    assert s[0, 0] == 3.0 and s[0, 1] == 4.0  # blocked: min(3, 4) = 3; after it, gap 1.5 > 1
    assert s[1, 0] == 3.0


def test_blocked_step_carries_responsiveness(oracle_lib):
    # Eq. 1 second case is R_c * delta_min: with rho = 1 at d = 0, R = 1 - 0.1
    r = race([0.0, 0.5], [10.0, 4.0], rho=[1.0, 0.5], L=100.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=2)
    s0 = float(steps_of(traj, [0.0, 0.5])[0, 0])
    assert abs(s0 - 0.9 * 4.0) < 1e-6


def test_nearest_in_front_not_first_or_farthest(oracle_lib):
    # c0 at 0 has c2 at 0.6 (prev 5) nearest in front and c1 at 0.8 (prev 2) farther:
    # i+ = c2, so S_c0 = min(10, 5) = 5, not min(10, 2) = 2
    r = race([0.0, 0.8, 0.6], [10.0, 2.0, 5.0], theta=[1.0, 0.0, 0.0], L=1000.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=1)
    assert float(steps_of(traj, [0.0, 0.8, 0.6])[0, 0]) == 5.0


def test_nearest_in_front_tie_takes_lowest_index(oracle_lib):
    # c1 and c2 both at 0.6: i+ = c1 (lowest index), prev 2 -> S_c0 = 2
    r = race([0.0, 0.6, 0.6], [10.0, 2.0, 5.0], theta=[1.0, 0.0, 0.0], L=1000.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=1)
    assert float(steps_of(traj, [0.0, 0.6, 0.6])[0, 0]) == 2.0
    r = race([0.0, 0.6, 0.6], [10.0, 5.0, 2.0], theta=[1.0, 0.0, 0.0], L=1000.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=1)
    assert float(steps_of(traj, [0.0, 0.6, 0.6])[0, 0]) == 5.0


def test_equal_positions_do_not_block(oracle_lib):
    # "in front" is strict: competitors level with each other run free
    r = race([0.0, 0.0], [10.0, 4.0], L=1000.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=1)
    assert list(steps_of(traj, [0.0, 0.0])[0]) == [10.0, 4.0]


def test_synchronous_update(oracle_lib):
    # c0 at 0 blocked by c1 at 0.5 reads c1's previous step (prev0 = 4), not the step c1
    # takes at the same time (6 here, prev0 given explicitly)
    r = race([0.0, 0.5], [10.0, 6.0], prev0=[10.0, 4.0], L=1000.0)
    w, steps, traj = oracle_lib.rollout(r, 0, 0, 0, traj_cap=1)
    assert list(steps_of(traj, [0.0, 0.5])[0]) == [4.0, 6.0]


def test_winner_is_earliest_crossing_not_farthest(oracle_lib):
    # L = 100: c0 at 89 steps 13 (lands at 102, tau = 11/13); c1 at 96 steps 5 (lands at
    # 101, tau = 4/5): c1 crossed first within the step
    r = race([89.0, 96.0], [13.0, 5.0], L=100.0)
    w, steps, _ = oracle_lib.rollout(r, 0, 0, 0)
    assert (w, steps) == (1, 1)


def test_exact_crossing_tie_takes_lowest_index(oracle_lib):
    r = race([95.0, 90.0], [5.0, 10.0], theta=[0.0, 0.0], L=100.0)  # both tau = 1
    assert oracle_lib.rollout(r, 0, 0, 0)[0] == 0
    r = race([90.0, 95.0], [10.0, 5.0], theta=[0.0, 0.0], L=100.0)
    assert oracle_lib.rollout(r, 0, 0, 0)[0] == 0


def test_finish_line_is_inclusive(oracle_lib):
    # Section 3: a competitor has finished once d_c >= L
    r = race([0.0], [50.0], L=100.0)
    assert oracle_lib.rollout(r, 0, 0, 0)[1] == 2


def test_step_limit_reports_status(oracle_lib):
    r = race([0.0], [1.0], L=100.0)
    counts, steps, st = oracle_lib.race_counts(r, 0, R=3, max_steps=10)
    assert st == oracle_lib.STEP_LIMIT and counts.sum() == 0 and steps == 30


# ------------------------------------------------------------------ noise-free closed form

def test_zero_noise_closed_form(oracle_lib):
    # sigma = 0, rho = 1/2, P = 1, theta = 0 (no blocking): every competitor moves exactly
    # mu_c per step and crosses L at real time (L - d0_c) / mu_c; the winner is its argmin
    # and wins every rollout.
    rng = np.random.default_rng(3)
    done = 0
    while done < 40:
        n = int(rng.integers(2, 9))
        L = 1000
        d0 = rng.integers(0, 900, n)
        mu = rng.integers(3, 30, n)
        times = [Fraction(int(L - a), int(m)) for a, m in zip(d0, mu)]
        srt = sorted(times)
        if srt[1] - srt[0] < Fraction(1, 100):
            continue  # keep away from near-ties
        want = times.index(srt[0])
        r = race(d0.astype(float), mu.astype(float), theta=[0.0] * n, L=float(L))
        counts, steps, st = oracle_lib.race_counts(r, 0, R=5)
        assert st == 0 and counts[want] == 5, (d0, mu, counts)
        assert steps == 5 * int(np.ceil(float(srt[0])))
        done += 1


# ------------------------------------------------------------------ exhaustive enumeration

ENUM_CASES = [
    # (L, d0, mu, sigma, P, theta)
    (12.0, [0.0, 0.0], [3.0, 3.0], [1.0, 2.0], None, [1.0, 1.0]),
    (16.0, [0.0, 1.0], [4.0, 3.0], [1.0, 1.5], None, [1.5, 1.0]),
    (14.0, [0.0, 0.5, 1.0], [3.0, 3.5, 2.5], [1.0, 1.5, 0.5], None, [1.0, 1.0, 1.0]),
    (13.0, [2.0, 0.0, 1.0], [3.0, 4.0, 3.5], [2.0, 1.0, 0.5], [1.0, 0.75, 1.0], [2.0, 0.5, 1.0]),
]


@pytest.mark.parametrize("case", range(len(ENUM_CASES)))
def test_two_point_races_match_exhaustive_enumeration(oracle_lib, case):
    L, d0, mu, sigma, P, theta = ENUM_CASES[case]
    exact = exact_win_probs(L, d0, mu, sigma, P=P, theta=theta)
    assert abs(exact.sum() - 1.0) < 1e-12
    R = 200000
    r = race(d0, mu, sigma, P=P, theta=theta, L=L, dist=2, R=R, race_id=case)
    counts, steps, st = oracle_lib.race_counts(r, 11)
    assert st == 0 and counts.sum() == R
    p = counts / R
    tol = 5 * np.sqrt(exact * (1 - exact) / R) + 1e-9
    assert np.all(np.abs(p - exact) <= tol), (p, exact)


def test_enumeration_sees_blocking(oracle_lib):
    # the enumerated cases do exercise Eq. 1's second case: with theta = 0 (no blocking)
    # the exact distribution of case 2 changes
    L, d0, mu, sigma, P, theta = ENUM_CASES[2]
    a = exact_win_probs(L, d0, mu, sigma, P=P, theta=theta)
    b = exact_win_probs(L, d0, mu, sigma, P=P, theta=[0.0] * 3)
    assert np.max(np.abs(a - b)) > 0.01


# ------------------------------------------------------------------ estimator invariants

def test_counts_sum_to_rollouts_and_probs(oracle_lib):
    from paper_2108_02419_gb300 import workloads as W

    b = W.single_race_start(rollouts=500)
    counts, steps, st = oracle_lib.race_counts(b.race(0), b.seed)
    assert st == 0 and counts.sum() == 500 and steps >= 500
    p, odds = oracle_lib.win_probs(counts, 500)
    assert abs(p.astype(np.float64).sum() - 1.0) < 1e-6
    assert np.all(odds[counts > 0] == np.float32(1.0) / p[counts > 0])
    assert np.all(np.isinf(odds[counts == 0]))


def test_identical_competitors_equal_chances(oracle_lib):
    n, R = 4, 20000
    r = race([0.0] * n, [16.0] * n, [1.0] * n, rho=[0.3] * n, L=300.0, R=R)
    counts, _, _ = oracle_lib.race_counts(r, 5)
    p = counts / R
    assert np.all(np.abs(p - 1 / n) <= 5 * np.sqrt((1 / n) * (1 - 1 / n) / R))


def test_relabelling_gives_same_distribution(oracle_lib):
    R = 20000
    base = dict(d0=[0.0, 3.0, 5.0], mu=[16.5, 16.0, 15.5], sigma=[1.5, 1.0, 0.7], rho=[0.2, 0.9, 0.5])
    perm = [2, 0, 1]
    a, _, _ = oracle_lib.race_counts(race(**base, L=400.0, R=R), 1)
    pb = {k: [v[i] for i in perm] for k, v in base.items()}
    b, _, _ = oracle_lib.race_counts(race(**pb, L=400.0, R=R), 1)
    pa, pbb = a / R, b[np.argsort(perm)] / R
    tol = 5 * np.sqrt(2 * pa * (1 - pa) / R) + 1e-9
    assert np.all(np.abs(pa - pbb) <= tol)


def test_monotone_in_speed_and_position(oracle_lib):
    R = 20000
    base = dict(d0=[0.0, 0.0, 0.0], mu=[16.0, 16.0, 16.0], sigma=[1.0, 1.0, 1.0])
    p0 = oracle_lib.race_counts(race(**base, L=400.0, R=R), 2)[0] / R
    faster = dict(base, mu=[16.3, 16.0, 16.0])
    p1 = oracle_lib.race_counts(race(**faster, L=400.0, R=R), 2)[0] / R
    ahead = dict(base, d0=[4.0, 0.0, 0.0])
    p2 = oracle_lib.race_counts(race(**ahead, L=400.0, R=R), 2)[0] / R
    sd = np.sqrt(0.25 / R)
    assert p1[0] > p0[0] + 5 * sd and p2[0] > p0[0] + 5 * sd


def test_rollouts_are_independent_of_batching(oracle_lib):
    # counter-based stream: rollouts [0, 300) equal [0, 100) + [100, 300)
    r = race([0.0, 2.0, 4.0], [16.0, 15.8, 15.5], [1.2, 1.0, 0.8], L=300.0, R=300)
    a, sa, _ = oracle_lib.race_counts(r, 3)
    b1, s1, _ = oracle_lib.race_counts(r, 3, R=100)
    b2, s2, _ = oracle_lib.race_counts(r, 3, R=200, k_begin=100)
    assert np.array_equal(a, b1 + b2) and sa == s1 + s2


def test_race_id_keys_the_stream(oracle_lib):
    r = race([0.0, 2.0, 4.0], [16.0, 15.8, 15.5], [1.2, 1.0, 0.8], L=300.0, R=2000)
    a, sa, _ = oracle_lib.race_counts(r, 3, r=0)
    b, sb, _ = oracle_lib.race_counts(r, 3, r=1)
    assert not (np.array_equal(a, b) and sa == sb)
