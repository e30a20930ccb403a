"""Float64 reference of the win-probability surrogate network (test infrastructure only).

The network maps a race state to a win-probability vector, permutation-equivariantly:

  per competitor c of a race (n competitors, track length L), features: the raw quantities
    [ d_c / L, (L - d_c) / 5000, mu_c - 16, sigma_c - 1, 2 rho_c - 1 ] and nine values derived
    from them per race (expected finish time and its spread, the lag behind the race's fastest
    expected finisher and its z-score, the gaps to the competitors ahead and behind, 1/n, and
    the two catch-up shares; see features()); the five-input network sees the raw five alone
  encoder (3 layers, width 128, ReLU):  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3)
  context: g = mean over the race's competitors of h3
  head:    u_c = relu(W4 [h3_c ; g] + b4)        (256 -> 128)
           logit_c = w5 . u_c + b5
  output:  q = softmax over the race's competitors of the logits
  loss:    cross-entropy against Monte Carlo win probabilities p: -sum_c p_c log q_c,
           averaged over the races of a batch.

Parameters live in one flat float vector in this order (row-major [out][in] matrices; W1 is
stored with its input dimension padded from 14 to 16 with zeros):
  W1 [128][16], b1 [128], W2 [128][128], b2, W3 [128][128], b3, W4 [128][256], b4, w5 [128], b5 [1].
W1's columns 14..15 multiply zero inputs (and columns 5..13 too in the five-input network).

With ``bf16=True`` the forward pass rounds to bfloat16 (round to nearest even) exactly where a
mixed-precision implementation keeps bfloat16 values: the weight matrices, the features, and
h1, h2, h3, the context g and u before they enter the next product; all sums are float64.
Without it everything is float64.  The backward pass is the exact derivative of the float64
forward (of the rounded inputs when bf16=True, with the roundings treated as identity).
"""
from __future__ import annotations

import numpy as np

H = 128
FIN = 14
KIN = 16
L_SCALE = 5000.0

SHAPES = [("W1", (H, KIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (H, 2 * H)), ("b4", (H,)), ("w5", (H,)), ("b5", (1,))]
N_PARAMS = int(sum(np.prod(s) for _, s in SHAPES))


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS, flat.size
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def features(d, L, mu, sigma, rho, race_off=None):
    """Input features of each competitor (float64), 16 columns.

    Columns 0..4 are the raw quantities [d/L, (L-d)/5000, mu-16, sigma-1, 2 rho-1].  With
    race_off given, columns 5..10 are derived from them per race:
      v = mu (1 + 0.1 (2 rho - 1) d/L)   expected speed (the responsiveness law averaged
                                          over the rest of the track)
      T = (L - d) / v                     expected steps to the line;  s = sigma sqrt(T) / v
      x5 = T / 100,  x6 = min(T - Tmin, 100) / 10,  x7 = s,
      x8 = min((T - Tmin) / sqrt(s^2 + s_min^2 + 0.01), 20) / 5,
      x9 = min(gap to the nearest competitor strictly ahead, 100) / 10 (100 when none),
      x10 = 1 / n,
      x11 = min(gap to the nearest competitor strictly behind, 100) / 10 (100 when none),
      x12 = min(g_a / (v - v_a) / T, 2) / 2 when the nearest competitor ahead (gap g_a, speed
            v_a) is slower, else 1: the share of its remaining race after which this competitor
            would catch it,
      x13 = min(g_b / (v_b - v) / T_b, 2) / 2 when the nearest competitor behind (gap g_b, speed
            v_b, time T_b) is faster, else 1,
    where Tmin is the race's least T and s_min the s of that competitor; "nearest" takes the
    lowest index among equal positions, like i+ of Eq. 1.  Columns 14..15 are zero."""
    d, L, mu, sigma, rho = (np.asarray(a, np.float64) for a in (d, L, mu, sigma, rho))
    x = np.zeros((d.size, KIN))
    frac = d / L
    x[:, 0] = frac
    x[:, 1] = (L - d) / L_SCALE
    x[:, 2] = mu - 16.0
    x[:, 3] = sigma - 1.0
    x[:, 4] = 2.0 * rho - 1.0
    if race_off is None:
        return x
    v = mu * (1.0 + 0.1 * (2.0 * rho - 1.0) * frac)
    T = (L - d) / v
    sd = sigma * np.sqrt(T) / v
    off = np.asarray(race_off, np.int64)
    for r in range(off.size - 1):
        a, b = off[r], off[r + 1]
        k = a + int(np.argmin(T[a:b]))
        lag = T[a:b] - T[k]
        x[a:b, 5] = T[a:b] / 100.0
        x[a:b, 6] = np.minimum(lag, 100.0) / 10.0
        x[a:b, 7] = sd[a:b]
        x[a:b, 8] = np.minimum(lag / np.sqrt(sd[a:b] ** 2 + sd[k] ** 2 + 0.01), 20.0) / 5.0
        for c in range(a, b):
            ia = ib = None
            for i in range(a, b):
                if d[i] > d[c] and (ia is None or d[i] < d[ia]):
                    ia = i
                if d[i] < d[c] and (ib is None or d[i] > d[ib]):
                    ib = i
            ga = d[ia] - d[c] if ia is not None else 100.0
            gb = d[c] - d[ib] if ib is not None else 100.0
            x[c, 9] = min(ga, 100.0) / 10.0
            x[c, 11] = min(gb, 100.0) / 10.0
            x[c, 12] = min(ga / (v[c] - v[ia]) / T[c], 2.0) / 2.0 if ia is not None and v[c] > v[ia] else 1.0
            x[c, 13] = min(gb / (v[ib] - v[c]) / T[ib], 2.0) / 2.0 if ib is not None and v[ib] > v[c] else 1.0
        x[a:b, 10] = 1.0 / (b - a)
    return x


def forward(params, x, race_off, bf16=False):
    """Forward pass over a CSR batch of races.  Returns (q, cache)."""
    p = unpack(params) if not isinstance(params, dict) else params
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    W1, W2, W3, W4 = (rnd(p[k]) for k in ("W1", "W2", "W3", "W4"))
    x = rnd(x)
    a1 = x @ W1.T + p["b1"]
    h1 = rnd(np.maximum(a1, 0.0))
    a2 = h1 @ W2.T + p["b2"]
    h2 = rnd(np.maximum(a2, 0.0))
    a3 = h2 @ W3.T + p["b3"]
    h3f = np.maximum(a3, 0.0)
    h3 = rnd(h3f)
    off = np.asarray(race_off, np.int64)
    sizes = np.diff(off)
    race_of = np.repeat(np.arange(sizes.size), sizes)
    gsum = np.zeros((sizes.size, H))
    np.add.at(gsum, race_of, h3)
    g_race = rnd(gsum / sizes[:, None])
    g = g_race[race_of]
    z = np.concatenate([h3, g], axis=1)
    a4 = z @ W4.T + p["b4"]
    u = np.maximum(a4, 0.0)
    ur = rnd(u)
    logit = ur @ p["w5"] + p["b5"][0]
    q = np.empty_like(logit)
    for r in range(sizes.size):
        s = slice(off[r], off[r + 1])
        e = np.exp(logit[s] - logit[s].max())
        q[s] = e / e.sum()
    cache = dict(x=x, W1=W1, W2=W2, W3=W3, W4=W4, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, g=g, z=z, a4=a4,
                 u=ur, logit=logit, q=q, off=off, sizes=sizes, race_of=race_of, p=p)
    return q, cache


def loss(params, x, race_off, target, bf16=False):
    q, _ = forward(params, x, race_off, bf16)
    n_races = len(race_off) - 1
    return float(-(np.asarray(target, np.float64) * np.log(np.maximum(q, 1e-300))).sum() / n_races)


def backward(params, x, race_off, target, bf16=False):
    """Gradient of the mean cross-entropy with respect to the flat parameter vector.

    With bf16=True the gradient activations entering each matrix product (du, and the
    gradients at the pre-activations of layers 3, 2, 1) are rounded to bfloat16 as well,
    as a mixed-precision backward pass does; bias gradients use the unrounded values."""
    q, c = forward(params, x, race_off, bf16)
    p = c["p"]
    rnd = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    n_races = c["sizes"].size
    t = np.asarray(target, np.float64)
    # softmax + cross-entropy per race: d loss / d logit_c = (q_c sum(t) - t_c) / n_races
    tsum = np.zeros(n_races)
    np.add.at(tsum, c["race_of"], t)
    dlogit = (q * tsum[c["race_of"]] - t) / n_races
    g = {}
    g["w5"] = c["u"].T @ dlogit
    g["b5"] = np.array([dlogit.sum()])
    du = np.outer(dlogit, p["w5"]) * (c["a4"] > 0)
    g["b4"] = du.sum(0)
    du = rnd(du)
    g["W4"] = du.T @ c["z"]
    dz = du @ c["W4"]
    dh3 = dz[:, :H].copy()
    dgr = np.zeros((n_races, H))
    np.add.at(dgr, c["race_of"], dz[:, H:])
    dh3 += (dgr / c["sizes"][:, None])[c["race_of"]]
    da3 = dh3 * (c["a3"] > 0)
    g["b3"] = da3.sum(0)
    da3 = rnd(da3)
    g["W3"] = da3.T @ c["h2"]
    da2 = (da3 @ c["W3"]) * (c["a2"] > 0)
    g["b2"] = da2.sum(0)
    da2 = rnd(da2)
    g["W2"] = da2.T @ c["h1"]
    da1 = (da2 @ c["W2"]) * (c["a1"] > 0)
    g["b1"] = da1.sum(0)
    da1 = rnd(da1)
    g["W1"] = da1.T @ c["x"]
    return pack(g)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights for the ReLU layers, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    p = {}
    p["W1"] = np.zeros((H, KIN))
    p["W1"][:, :FIN] = rng.uniform(-1, 1, (H, FIN)) * np.sqrt(6.0 / FIN)
    p["W2"] = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    p["W3"] = rng.uniform(-1, 1, (H, H)) * np.sqrt(6.0 / H)
    p["W4"] = rng.uniform(-1, 1, (H, 2 * H)) * np.sqrt(6.0 / (2 * H))
    p["w5"] = rng.uniform(-1, 1, H) * np.sqrt(3.0 / H)
    for b in ("b1", "b2", "b3", "b4"):
        p[b] = np.zeros(H)
    p["b5"] = np.zeros(1)
    return pack(p)
