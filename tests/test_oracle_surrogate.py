"""Pins of the float64 surrogate reference: finite differences for the backward pass,
structural facts of the forward pass (softmax, equivariance, symmetric inputs), and the
bfloat16 rounding against its definition."""
import numpy as np
import pytest

from oracle import surrogate_ref as S


def _batch(seed, sizes):
    rng = np.random.default_rng(seed)
    n = int(np.sum(sizes))
    off = np.concatenate([[0], np.cumsum(sizes)])
    L = np.repeat(np.full(len(sizes), 5000.0), sizes)
    d = L - rng.uniform(100, 5000, n)
    x = S.features(d, L, rng.uniform(15, 17, n), rng.uniform(0.5, 1.5, n), rng.uniform(0, 1, n))
    t = np.empty(n)
    for r in range(len(sizes)):
        w = rng.dirichlet(np.ones(sizes[r]))
        t[off[r]:off[r + 1]] = w
    return x, off, t


def test_param_count():
    assert S.N_PARAMS == 128 * 16 + 128 + 2 * (128 * 128 + 128) + 128 * 256 + 128 + 128 + 1


def test_finite_differences():
    x, off, t = _batch(1, [3, 5, 2])
    params = S.init_params(3)
    params[S.N_PARAMS - 1] = 0.1
    g = S.backward(params, x, off, t)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(S.N_PARAMS, 60, replace=False), [S.N_PARAMS - 1, 0, 1, 2, 3, 4]])
    for i in idx:
        e = np.zeros(S.N_PARAMS)
        h = 1e-6 * max(1.0, abs(params[i]))
        e[i] = h
        num = (S.loss(params + e, x, off, t) - S.loss(params - e, x, off, t)) / (2 * h)
        assert abs(num - g[i]) <= 1e-6 * max(1e-3, abs(num)) + 1e-9, (i, num, g[i])


def test_softmax_per_race_and_equivariance():
    x, off, t = _batch(2, [4, 7])
    params = S.init_params(5)
    q, _ = S.forward(params, x, off)
    assert abs(q[:4].sum() - 1) < 1e-12 and abs(q[4:].sum() - 1) < 1e-12
    perm = np.concatenate([[2, 0, 3, 1], 4 + np.array([6, 5, 4, 3, 2, 1, 0])])
    q2, _ = S.forward(params, x[perm], off)
    assert np.allclose(q2, q[perm], atol=1e-14)
    # a race's output does not depend on other races in the batch
    q3, _ = S.forward(params, x[:4], off[:2])
    assert np.allclose(q3, q[:4], atol=1e-14)


def test_identical_competitors_get_equal_probabilities():
    x = np.tile(S.features([1000.0], [5000.0], [16.0], [1.0], [0.5]), (6, 1))
    q, _ = S.forward(S.init_params(6), x, [0, 6])
    assert np.allclose(q, 1 / 6, atol=1e-14)


def test_zero_head_gives_uniform():
    params = S.unpack(S.init_params(7))
    params["w5"][:] = 0.0
    x, off, t = _batch(3, [5])
    q, _ = S.forward(params, x, off)
    assert np.allclose(q, 0.2, atol=1e-15)


def test_bf16_rounding_definition():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-30, 0.0], np.float32)
    r = S.bf16_round(vals)
    # bfloat16 keeps 8 significant bits: the result has at most 8 and is the nearest such value
    for v, rv in zip(vals.astype(np.float64), r):
        if v == 0:
            assert rv == 0
            continue
        e = np.floor(np.log2(abs(v)))
        ulp = 2.0 ** (e - 7)
        assert abs(rv - v) <= ulp / 2 + 1e-300
        assert (rv / ulp) == np.round(rv / ulp)
    assert S.bf16_round(np.float32(1.005859375)) == 1.0078125  # tie 1 + 1.5/256 -> even


def test_bf16_backward_close_to_float64():
    x, off, t = _batch(8, [6, 3, 9])
    params = S.init_params(9)
    g64 = S.backward(params, x, off, t)[:-1]  # b5's gradient is zero when targets sum to 1
    g16 = S.backward(params, x, off, t, bf16=True)[:-1]
    cos = g16 @ g64 / (np.linalg.norm(g16) * np.linalg.norm(g64))
    assert cos > 0.97, cos  # same direction; bfloat16 products cancel less exactly than float64


def test_derived_features_worked_example():
    # race of three on L = 1000: c0 at 0 (mu 10, rho 1/2), c1 at 500 (mu 10, rho 1), c2 at 520
    L = np.full(3, 1000.0)
    d = np.array([0.0, 500.0, 520.0])
    mu = np.array([10.0, 10.0, 8.0])
    sig = np.array([1.0, 2.0, 0.0])
    rho = np.array([0.5, 1.0, 0.5])
    x = S.features(d, L, mu, sig, rho, [0, 3])
    T = np.array([100.0, 500.0 / 10.5, 60.0])  # v = mu (1 + 0.1 (2 rho - 1) d / L)
    assert np.allclose(x[:, 5], T / 100)
    assert np.allclose(x[:, 6], (T - T[1]) / 10)          # c1 has the least expected finish time
    sd = sig * np.sqrt(T) / np.array([10.0, 10.5, 8.0])
    assert np.allclose(x[:, 7], sd)
    assert x[1, 8] == 0.0 and np.isclose(x[0, 8], min((T[0] - T[1]) / np.sqrt(sd[0] ** 2 + sd[1] ** 2 + 0.01), 20) / 5)
    assert np.allclose(x[:, 9], [10.0, 2.0, 10.0])        # gaps ahead: 500 -> capped 100, 20, none -> 100
    assert np.allclose(x[:, 10], 1 / 3)
    assert np.allclose(x[:, 11], [10.0, 10.0, 2.0])       # gaps behind: none, 500 -> 100, 20
    catch = 20.0 / (10.5 - 8.0) / T[1]                     # c1 closes 20 units at 2.5 units a step
    assert np.allclose(x[:, 12], [1.0, catch / 2, 1.0])   # c0 is slower than c1; c2 leads
    assert np.allclose(x[:, 13], [1.0, 1.0, catch / 2])   # only c2 has a faster competitor behind
    assert np.all(x[:, 14:] == 0)
    # relabelling the competitors relabels the features
    perm = [2, 0, 1]
    xp = S.features(d[perm], L, mu[perm], sig[perm], rho[perm], [0, 3])
    assert np.allclose(xp, x[perm])


def test_worked_example_by_hand():
    """A two-competitor race through hand-set weights, computed by hand.

    A: d/L = 0.2, mu - 16 = 0.5;  B: d/L = 0.6, mu - 16 = -0.5 (sigma 1, rho 1/2: columns 3, 4 zero).
    W1 picks column 0 into unit 0 and column 2 into unit 1; W2, W3 pass units 0, 1 on:
      h3_A = (0.2, 0.5), h3_B = (0.6, 0)             (ReLU clips B's -0.5)
      g = mean = (0.4, 0.25)
    W4 row 0 = 3 h3_0 - 2 g_0, row 1 = 2 h3_1 + g_1 (b4 = 0):
      u_A = (relu(0.6 - 0.8), relu(1.0 + 0.25)) = (0, 1.25)
      u_B = (relu(1.8 - 0.8), relu(0 + 0.25))   = (1.0, 0.25)
    w5 = (1.5, 1.0), b5 = 0.2:  logit_A = 1.25 + 0.2 = 1.45, logit_B = 1.5 + 0.25 + 0.2 = 1.95
      q_A = 1 / (1 + e^0.5), q_B = 1 / (1 + e^-0.5).
    Pooling by sum (g = (0.8, 0.5)) would give logits 1.7 and 1.0, concatenating [g; h3]
    instead of [h3; g] or dropping a ReLU other values still."""
    p = {k: np.zeros(shp) for k, shp in S.SHAPES}
    p["W1"][0, 0] = 1.0
    p["W1"][1, 2] = 1.0
    for k in ("W2", "W3"):
        p[k][0, 0] = p[k][1, 1] = 1.0
    p["W4"][0, 0], p["W4"][0, 128] = 3.0, -2.0
    p["W4"][1, 1], p["W4"][1, 129] = 2.0, 1.0
    p["w5"][0], p["w5"][1] = 1.5, 1.0
    p["b5"][0] = 0.2
    x = S.features([1000.0, 3000.0], [5000.0, 5000.0], [16.5, 15.5], [1.0, 1.0], [0.5, 0.5])
    q, c = S.forward(S.pack(p), x, [0, 2])
    assert np.allclose(c["g"][0, :2], [0.4, 0.25], atol=1e-15)
    assert np.allclose(c["logit"], [1.45, 1.95], atol=1e-14)
    assert np.allclose(q, [1.0 / (1.0 + np.exp(0.5)), 1.0 / (1.0 + np.exp(-0.5))], atol=1e-15)
