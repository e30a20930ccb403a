"""Pins of the oracle's random step generator delta(v_c) (Section 3: S_c is stochastic).

- Philox4x32-10 against the published known-answer vectors (tests/golden).
- log and sin/cos(2 pi u) against float64 libm over EVERY input the generator can produce
  (2^24 values each), within 2 units in the last place of binary32.
- The Box-Muller output against the textbook transform evaluated in float64 on the same
  Philox words, and its distribution (moments, Kolmogorov-Smirnov, pair independence).
- The uniform and two-point variants' moments.
"""
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers(oracle_lib):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = oracle_lib.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_counter_sensitivity(oracle_lib):
    # every counter and key word changes every output word (avalanche, no ignored input)
    base = oracle_lib.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        ctr = [1, 2, 3, 4]
        ctr[i] ^= 1
        out = oracle_lib.philox4x32_10(ctr, [5, 6])
        assert np.all(out != base)
    for i in range(2):
        key = [5, 6]
        key[i] ^= 1
        out = oracle_lib.philox4x32_10([1, 2, 3, 4], key)
        assert np.all(out != base)


def _ulp_err(got, ref):
    ref32 = np.abs(ref).astype(np.float32)
    ulp = np.spacing(ref32).astype(np.float64)
    return np.abs(got.astype(np.float64) - ref) / ulp


def test_log_all_inputs_within_2ulp(oracle_lib):
    # the Box-Muller radius takes log of u1 = m * 2^-24, m = 1 .. 2^24: test every one
    m = np.arange(1, (1 << 24) + 1, dtype=np.float64)
    u1 = (m * 2.0 ** -24).astype(np.float32)
    assert np.all(u1.astype(np.float64) == m * 2.0 ** -24)  # the conversion is exact
    y = oracle_lib.log_f32(u1)
    ref = np.log(u1.astype(np.float64))
    assert y[-1] == 0.0  # log 1 = 0 exactly
    err = _ulp_err(y[:-1], ref[:-1])
    assert err.max() <= 2.0, err.max()


def test_log_other_binades(oracle_lib):
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(-80, 80, 200000)).astype(np.float32)
    y = oracle_lib.log_f32(x)
    ref = np.log(x.astype(np.float64))
    nz = np.abs(ref) > 1e-30
    assert _ulp_err(y[nz], ref[nz]).max() <= 2.0


def test_sincos_all_inputs_within_2ulp(oracle_lib):
    m = np.arange(0, 1 << 24, dtype=np.uint32)
    s, c = oracle_lib.sincos2pi(m)
    ang = 2.0 * np.pi * m.astype(np.float64) * 2.0 ** -24
    for got, ref in ((s, np.sin(ang)), (c, np.cos(ang))):
        zero = np.abs(ref) < 1e-12  # u in {0, 1/4, 1/2, 3/4}
        assert zero.sum() == 2
        assert np.all(got[zero] == 0.0)
        assert _ulp_err(got[~zero], ref[~zero]).max() <= 2.0
    # quadrant points are exact
    assert (s[0], c[0]) == (0.0, 1.0)
    assert (s[1 << 22], c[1 << 22]) == (1.0, 0.0)
    assert (s[1 << 23], c[1 << 23]) == (0.0, -1.0)
    assert (s[3 << 22], c[3 << 22]) == (-1.0, 0.0)


def test_box_muller_matches_textbook_on_philox_words(oracle_lib):
    # z(r, k, t, c) = sqrt(-2 ln u1) * (cos | sin)(2 pi u2), u1, u2 from the Philox block
    # with counter (k, t >> 2, c, r): pair (w0, w1) for t mod 4 in {0, 1}, (w2, w3) for
    # {2, 3}; cos for even t, sin for odd t; u1 = ((wa >> 8) + 1) 2^-24, u2 = (wb >> 8) 2^-24.
    seed = 0x0123456789ABCDEF
    rng = np.random.default_rng(2)
    for _ in range(400):
        r, k, c = (int(x) for x in rng.integers(0, 1 << 31, 3))
        t = int(rng.integers(0, 1 << 20))
        w = oracle_lib.philox4x32_10([k, t >> 2, c, r], [seed & 0xFFFFFFFF, seed >> 32])
        wa, wb = (w[0], w[1]) if ((t >> 1) & 1) == 0 else (w[2], w[3])
        u1 = ((int(wa) >> 8) + 1) * 2.0 ** -24
        u2 = (int(wb) >> 8) * 2.0 ** -24
        rad = np.sqrt(-2.0 * np.log(u1))
        want = rad * (np.cos(2 * np.pi * u2) if t % 2 == 0 else np.sin(2 * np.pi * u2))
        got = oracle_lib.z(0, seed, r, k, t, c)
        assert abs(got - want) <= 4e-7 * max(rad, 1e-3) + 1e-7, (got, want)


def test_normal_distribution(oracle_lib):
    z = oracle_lib.z_block(0, 0, 7, 0, 250000, 8, 3).astype(np.float64)
    x = z.ravel()
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(stats.skew(x)) < 5 * np.sqrt(6.0 / n)
    assert abs(stats.kurtosis(x)) < 5 * np.sqrt(24.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    assert np.abs(x).max() <= 5.77  # sqrt(-2 ln 2^-24) bounds |z|
    # independence: within a rollout across steps (pairs and across Philox blocks)
    for lag in (1, 2, 4):
        rho = np.corrcoef(z[:, :-lag].ravel(), z[:, lag:].ravel())[0, 1]
        assert abs(rho) < 5 / np.sqrt(z[:, lag:].size)
    # across competitors and across races at the same (k, t)
    z2 = oracle_lib.z_block(0, 0, 7, 0, 250000, 8, 4).astype(np.float64)
    z3 = oracle_lib.z_block(0, 0, 8, 0, 250000, 8, 3).astype(np.float64)
    assert abs(np.corrcoef(x, z2.ravel())[0, 1]) < 5 / np.sqrt(n)
    assert abs(np.corrcoef(x, z3.ravel())[0, 1]) < 5 / np.sqrt(n)


def test_uniform_and_two_point(oracle_lib):
    u = oracle_lib.z_block(1, 5, 0, 0, 200000, 8, 0).astype(np.float64).ravel()
    n = u.size
    assert u.min() >= -np.sqrt(3) - 1e-6 and u.max() < np.sqrt(3) + 1e-6
    assert abs(u.mean()) < 5 / np.sqrt(n)
    assert abs(u.var() - 1.0) < 5 * np.sqrt(0.8 / n)
    assert stats.kstest(u, "uniform", args=(-np.sqrt(3), 2 * np.sqrt(3))).pvalue > 1e-4
    b = oracle_lib.z_block(2, 5, 0, 0, 200000, 8, 0).astype(np.float64)
    assert set(np.unique(b)) == {-1.0, 1.0}
    assert abs(b.mean()) < 5 / np.sqrt(b.size)
    rho = np.corrcoef(b[:, :-1].ravel(), b[:, 1:].ravel())[0, 1]
    assert abs(rho) < 5 / np.sqrt(b.size)


@pytest.mark.parametrize("dist", [0, 1, 2])
def test_stream_keyed_by_all_four_coordinates(oracle_lib, dist):
    base = oracle_lib.z(dist, 9, 1, 2, 3, 4)
    others = [oracle_lib.z(dist, 9, 1 + 1, 2, 3, 4), oracle_lib.z(dist, 9, 1, 2 + 1, 3, 4),
              oracle_lib.z(dist, 9, 1, 2, 3, 4 + 1), oracle_lib.z(dist, 10, 1, 2, 3, 4)]
    if dist == 2:
        # two values only: check over many draws instead
        a = oracle_lib.z_block(dist, 9, 1, 0, 4000, 4, 4)
        b = oracle_lib.z_block(dist, 9, 2, 0, 4000, 4, 4)
        assert (a != b).mean() > 0.4
    else:
        assert all(o != base for o in others)


def test_log_constants_are_the_committed_fit():
    # oracle/fit_log.py reproduces the ten binary32 coefficients of the log polynomial
    from oracle import fit_log

    assert fit_log.main(["--check"]) == 0
