"""The budget rule of the surrogate's two-stage Monte Carlo fallback (host code of the C-ABI
library, no GPU needed): hand-worked values, its caps, and the property it exists for -- with
the budget it picks, every probability of the race has a standard deviation of at most about
max_sd."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def bbe():
    from paper_2108_02419_gb300 import bbe as B
    from paper_2108_02419_gb300 import build

    build.build()
    return B


SD = 0.01 / 4.5


def test_decided_race_stays_at_the_pilot(bbe):
    # all 1000 pilot rollouts won by one competitor: q = 1 - 3e-3, v = 0.002991, v / SD^2 = 606 < pilot
    assert bbe.bbe_surrogate_fallback_budget([1000, 0, 0], 1000, 50000, SD) == 1000


def test_even_contest_takes_the_cap_or_the_variance_bound(bbe):
    # p = 1/2 exactly: v = 1/4, budget = ceil(0.25 / SD^2) = ceil(50625.000..) (or the cap)
    need = math.ceil(0.25 / SD**2)
    assert bbe.bbe_surrogate_fallback_budget([500, 500], 1000, 10**6, SD) == need
    assert bbe.bbe_surrogate_fallback_budget([500, 500], 1000, 50000, SD) == 50000


def test_hand_worked_long_shot(bbe):
    # p = 0.1 of 1000: h = 3 sqrt(0.09 / 1000) = 0.0284605, q = 0.1284605, v = 0.1119585
    p, R1 = 0.1, 1000
    h = 3 * math.sqrt(p * (1 - p) / R1)
    q = p + h
    assert abs(q - 0.12846050) < 1e-7
    want = math.ceil(q * (1 - q) / 0.005**2)
    assert want == 4479
    assert bbe.bbe_surrogate_fallback_budget([100, 900], R1, 10**6, 0.005) == max(
        want, math.ceil(0.9 * 0.1 / 0.005**2))  # competitor 2 (p = 0.9) is the mirror image


def test_budget_is_within_pilot_and_cap_and_monotone(bbe):
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(1, 25))
        R1 = int(rng.integers(1, 5000))
        cap = R1 + int(rng.integers(0, 100000))
        c = rng.multinomial(R1, rng.dirichlet(np.ones(n) * 0.3))
        sd = float(rng.uniform(1e-3, 0.05))
        b = bbe.bbe_surrogate_fallback_budget(c, R1, cap, sd)
        assert R1 <= b <= cap
        assert bbe.bbe_surrogate_fallback_budget(c, R1, cap, sd / 2) >= b  # tighter target, no fewer
        assert bbe.bbe_surrogate_fallback_budget(c, R1, cap + 1000, sd) >= b


def test_single_competitor_needs_no_more_than_the_pilot(bbe):
    assert bbe.bbe_surrogate_fallback_budget([37], 37, 1000, 1e-3) == 37


def test_chosen_budget_meets_the_spread_target(bbe):
    # pilot counts drawn from known probabilities; the true standard deviation at the budget
    # stays within 10 % of max_sd in at least 99 % of draws (three standard errors of slack)
    rng = np.random.default_rng(11)
    R1, cap, ok, trials = 2000, 10**7, 0, 0
    for _ in range(300):
        n = int(rng.integers(2, 21))
        p = rng.dirichlet(np.ones(n) * float(rng.choice([0.1, 0.5, 2.0])))
        c = rng.multinomial(R1, p)
        b = bbe.bbe_surrogate_fallback_budget(c, R1, cap, SD)
        sd = math.sqrt(float(np.max(p * (1 - p))) / b)
        ok += sd <= 1.1 * SD
        trials += 1
    assert ok >= 0.99 * trials


def test_bad_arguments_are_refused(bbe):
    for args in (([], 10, 100, SD), ([1, 2], 0, 100, SD), ([1, 2], 10, 5, SD), ([1, 2], 10, 100, 0.0),
                 ([1, 2], 10, 100, 0.7)):
        with pytest.raises(bbe.BbeError):
            bbe.bbe_surrogate_fallback_budget(*args)
