"""Pins of the oracle's time law of responsiveness (Eq. 1's R_c(t, d), Section 3: a competitor
that starts fast and fades, or starts slowly and finishes strongly).  Reading: R_c =
1 + kappa (2 rho_c - 1) (u - 1/2) with u = min(1, (t0 + t) / T), the fraction of the race's
expected duration T elapsed; t0 is the steps elapsed before the state (a mid-race snapshot),
t the step of the dry-run.

The pins do not retype the law's binary32 operations.  (1) A noise-free race whose inputs make
every quantity a dyadic rational (kappa (2 rho - 1) = +-1/8, T = 64, mu = 16, integer t0) is
simulated in exact rational arithmetic from the law's mathematical statement; the oracle must
give its finishing step and winner.  (2) Continuing a noise-free race from a mid-race snapshot
with elapsed time s must reproduce the uninterrupted race.  (3) rho = 1/2 makes the law
irrelevant (R = 1 under both laws)."""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from paper_2108_02419_gb300 import workloads as W

RHO_UP, RHO_DOWN = 0.8125, 0.1875  # kappa (2 rho - 1) = +1/8 and -1/8 exactly in binary32


def test_dyadic_inputs_are_exact():
    kappa = np.float32(0.2)
    for rho, want in ((RHO_UP, 0.125), (RHO_DOWN, -0.125)):
        assert kappa * (np.float32(2.0) * np.float32(rho) - np.float32(1.0)) == np.float32(want)


def exact_race(d0, krs, mu, T, t0, L):
    """The time law in exact arithmetic: returns (finishing step count, winner)."""
    d = [F(x) for x in d0]
    t = 0
    while True:
        u = min(F(1), F(t0 + t, T))
        S = [F(mu) * (1 + kr * (u - F(1, 2))) for kr in krs]
        dn = [a + b for a, b in zip(d, S)]
        fin = [c for c in range(len(d)) if dn[c] >= L]
        if fin:
            tau = {c: (F(L) - d[c]) / S[c] for c in fin}
            best = min(tau.values())
            return t + 1, min(c for c in fin if tau[c] == best)
        d = dn
        t += 1


@pytest.mark.parametrize("t0", [0, 7, 30, 64, 100])
@pytest.mark.parametrize("L", [1000.0, 1100.0, 1640.0])
def test_noise_free_closed_form(t0, L):
    # a (closer, rho 0.8125) starts behind b (fader, rho 0.1875); theta = 0: no blocking
    d0, mu, T = [0.0, 40.0], 16.0, 64.0
    want_steps, want_winner = exact_race(d0, [F(1, 8), F(-1, 8)], mu, 64, t0, L)
    rb = W.from_arrays([2], L, 50, d0, [mu, mu], [0.0, 0.0], [RHO_UP, RHO_DOWN], theta=[0.0, 0.0], seed=3)
    rb = W.with_time_law(rb, float(t0), T)
    counts, steps, st = oracle.batch_counts(rb)
    assert st == 0
    assert counts[want_winner] == 50 and counts.sum() == 50
    assert steps[0] == 50 * want_steps


def test_law_differs_from_position_law():
    # the same inputs under the position law finish differently (the closed-form pin would not
    # pass by accident with the wrong law): another winner and another finishing step
    d0, mu = [0.0, 40.0], 16.0
    rb = W.from_arrays([2], 1640.0, 10, d0, [mu, mu], [0.0, 0.0], [RHO_UP, RHO_DOWN], theta=[0.0, 0.0], seed=3)
    c_pos, s_pos, _ = oracle.batch_counts(rb)
    c_time, s_time, _ = oracle.batch_counts(W.with_time_law(rb, 30.0, 64.0))
    assert c_pos[1] == 10 and c_time[0] == 10 and s_pos[0] != s_time[0]


@pytest.mark.parametrize("s", [1, 5, 13, 40])
def test_snapshot_continues_the_race(s):
    # noise-free, with blocking (theta 3): the state after s steps, with elapsed time s and the
    # last steps as previous steps, finishes exactly where the whole race does
    rng = np.random.default_rng(8)
    n = 6
    race = dict(n=n, L=1500.0, d0=np.sort(rng.uniform(0, 60, n)).astype(np.float32),
                mu=rng.uniform(15, 17, n).astype(np.float32), sigma=np.zeros(n, np.float32),
                rho=rng.uniform(0, 1, n).astype(np.float32), P=np.ones(n, np.float32),
                theta=np.full(n, 3.0, np.float32), prev0=None, dist=0, law=1, t0=0.0, T=90.0)
    d_traj, s_traj, _, _ = oracle.trajectory(race, seed=1, r=0, k=0)
    w_full, st_full, _ = oracle.rollout(race, seed=1, r=0, k=0)
    assert s < st_full
    snap = dict(race, d0=d_traj[s - 1].copy(), prev0=s_traj[s - 1].copy(), t0=float(s))
    w, st, _ = oracle.rollout(snap, seed=1, r=0, k=3)
    assert (w, st) == (w_full, st_full - s)


def test_neutral_responsiveness_ignores_the_law():
    rb = W.uneven_batch(seed=21, n_races=6, rollouts=300)
    rb.rho[:] = 0.5
    want = oracle.batch_counts(rb)
    got = oracle.batch_counts(W.with_time_law(rb, 12.0, 250.0))
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_fader_and_closer_swap_roles_with_time():
    # equal in everything but rho; late in the race (u held at 1) the closer is faster, early
    # (u near 0) the fader is
    rb = W.from_arrays([2], 600.0, 4000, [0.0, 0.0], [16.0, 16.0], [1.0, 1.0], [1.0, 0.0], seed=5)
    late, _, _ = oracle.batch_counts(W.with_time_law(rb, 1000.0, 100.0))
    early, _, _ = oracle.batch_counts(W.with_time_law(rb, 0.0, 10000.0))
    assert late[0] > 3000 and early[1] > 3000
