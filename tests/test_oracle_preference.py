"""Pins of the preference-vector law P_c(f_r, p_c) (Section 3; this library's reading
P_c = prod_k (1 - w_k min(1, |f_r,k - p_c,k|)))."""
import numpy as np

import oracle


def test_hand_worked():
    P = oracle.preference([0, 2, 3], [[0.5, 0.0], [1.0, 1.0]], [[0.5, 0.0], [0.0, 1.0], [0.25, 2.0]], [1.0, 0.5])
    # perfect match; (1 - 0.5)(1 - 0.5 * 1); (1 - 0.75)(1 - 0.5 * min(1, 1))
    assert list(P) == [1.0, 0.25, 0.125]


def test_invariants():
    rng = np.random.default_rng(4)
    off = np.array([0, 3, 7, 12], np.int32)
    f = rng.uniform(0, 1, (3, 5)).astype(np.float32)
    p = rng.uniform(-1, 2, (12, 5)).astype(np.float32)
    w = rng.uniform(0, 1, 5).astype(np.float32)
    P = oracle.preference(off, f, p, w)
    assert np.all((P >= 0) & (P <= 1))
    assert np.all(oracle.preference(off, f, p, np.zeros(5, np.float32)) == 1.0)       # no sensitivity
    same = np.repeat(f, np.diff(off), axis=0)
    assert np.all(oracle.preference(off, f, same, w) == 1.0)                           # perfect match
    # one factor: the closed form 1 - w min(1, |f - p|)
    P1 = oracle.preference(off, f[:, :1], p[:, :1], w[:1])
    want = 1 - w[0].astype(np.float64) * np.minimum(1, np.abs(np.repeat(f[:, 0], np.diff(off)).astype(np.float64) - p[:, 0]))
    assert np.allclose(P1, want, rtol=0, atol=2e-7)
    # a larger mismatch on one factor never raises P
    p2 = p.copy()
    p2[:, 2] += 0.3
    P2 = oracle.preference(off, f, p2, w)
    far = np.abs(np.repeat(f[:, 2], np.diff(off)) - p2[:, 2]) >= np.abs(np.repeat(f[:, 2], np.diff(off)) - p[:, 2])
    assert np.all(P2[far] <= P[far])
