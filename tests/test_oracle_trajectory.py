"""Pins of the oracle's full-race trajectory (Section 3: the race runs until its last
competitor crosses) and of the rule-based bettors' reference predictions (Section 4)."""
import numpy as np
import pytest

import oracle
from oracle import bettors as B
from tests.test_oracle_race import race


def test_zero_noise_trajectory_is_arithmetic(oracle_lib):
    # sigma = 0, rho = 1/2, P = 1, theta = 0: d_c(t) = d0_c + t mu_c exactly, until the last
    # competitor crosses
    d0 = np.array([0.0, 10.0, 3.0])
    mu = np.array([5.0, 4.0, 6.0])
    r = race(d0, mu, theta=[0.0] * 3, L=100.0)
    pos, stp, T, st = oracle.trajectory(r, 0, 0, 0)
    want_T = int(max(np.ceil((100.0 - d0) / mu)))
    assert st == 0 and T == want_T == 23
    t = np.arange(1, T + 1)[:, None]
    assert np.array_equal(pos, (d0 + t * mu).astype(np.float32))
    assert np.all(stp == mu.astype(np.float32))


def test_trajectory_extends_the_first_finisher_rollout_and_gives_the_order(oracle_lib):
    from paper_2108_02419_gb300 import workloads as W

    b = W.uneven_batch(seed=31, n_races=5, n_lo=2, n_hi=8, rollouts=3)
    for r in range(b.n_races):
        rc = b.race(r)
        for k in range(3):
            pos, stp, T, st = oracle.trajectory(rc, b.seed, r, k)
            w, ws, traj = oracle.rollout(rc, b.seed, r, k, traj_cap=100000)
            assert st == 0 and np.array_equal(pos[:ws], traj)
            assert np.all(pos[-1] >= rc["L"]) and not np.all(pos[-2] >= rc["L"])
            order, osteps, _ = oracle.rollout_order(rc, b.seed, r, k, rc["n"])
            assert osteps == T and order[0] == w
            # the order follows each competitor's first step across the line, then tau
            prev = np.vstack([rc["d0"][None, :], pos[:-1]])
            cross = [int(np.argmax(pos[:, c] >= rc["L"])) for c in range(rc["n"])]
            tau = [np.float32(np.float32(rc["L"]) - prev[cross[c], c]) / stp[cross[c], c] for c in range(rc["n"])]
            assert list(order) == sorted(range(rc["n"]), key=lambda c: (cross[c], tau[c], c))


def test_step_limit(oracle_lib):
    r = race([0.0, 1.0], [1.0, 1.0], sigma=[0.1, 0.1], L=1000.0)
    _, _, T, st = oracle.trajectory(r, 0, 0, 0, max_steps=50)
    assert T == 50 and st == oracle.STEP_LIMIT


# ------------------------------------------------------------------ rule-based bettors

def test_leader_and_underdog_hand_worked():
    d = np.array([5.0, 9.0, 9.0, 3.0], np.float32)
    assert B.leader(d) == 1                      # equal leaders: lower index
    assert B.underdog(d, 1.0) == 2               # P2 level with P1: within any positive gap
    assert B.underdog(d, 0.0) == 1               # gap 0: never the underdog
    d2 = np.array([5.0, 9.0, 7.5, 3.0], np.float32)
    assert B.underdog(d2, 1.5) == 1              # distance exactly D: back to the leader
    assert B.underdog(d2, 1.6) == 2
    assert B.underdog(np.array([4.0], np.float32), 10.0) == 0


def test_linex_hand_worked():
    # L 100; positions 80 and 90; recent steps 5,5 and 2,3: times 20/5 = 4 and 10/2.5 = 4 -> tie,
    # lower index; with a window of 1 the second competitor's speed is 3: 10/3 < 4
    d = np.array([80.0, 90.0], np.float32)
    steps = np.array([[9.0, 9.0], [5.0, 2.0], [5.0, 3.0]], np.float32)
    assert B.linex(d, steps, 3, 2, 100.0, [1.0, 1.0]) == 0
    assert B.linex(d, steps, 3, 1, 100.0, [1.0, 1.0]) == 1
    # the window reaches back past the start: all three steps (mean 19/3 and 14/3)
    assert B.linex(d, steps, 3, 10, 100.0, [1.0, 1.0]) == 1
    # at the start the previous-step inputs are the speeds
    assert B.linex(np.array([0.0, 0.0], np.float32), steps, 0, 5, 100.0, [4.0, 5.0]) == 1


def test_zero_intelligence_is_uniform_and_reproducible():
    picks = [B.zero_intelligence(5, 7, s, 3) for s in range(20000)]
    assert picks[:50] == [B.zero_intelligence(5, 7, s, 3) for s in range(50)]
    freq = np.bincount(picks, minlength=5) / len(picks)
    assert np.all(np.abs(freq - 0.2) < 5 * np.sqrt(0.16 / len(picks)))
    assert picks != [B.zero_intelligence(5, 7, s, 4) for s in range(20000)]
