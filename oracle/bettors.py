"""Rule-based bettors of the BBE model, plain reference predictions of the winner from a
race's trajectory (test infrastructure only, like the rest of this package).

Section 4 lists the bettor classes; the ones that predict from the race so far are:
  LW     Leader Wins: the competitor currently in the lead wins;
  UD     Underdog: the second-placed competitor wins while its distance to the leader is below
         a threshold D, otherwise the leader;
  LinEx  Linear Extrapolator: each competitor's speed is the mean of its step sizes over the
         last N time steps, assumed constant for the rest of the race; the competitor reaching
         the line first wins;
  ZI     Zero Intelligence: a competitor chosen at random.
Readings where the paper is silent: equal positions or equal extrapolated times go to the
lower index; LinEx at the start (no step yet) uses each competitor's previous-step input;
ZI draws (w0 * n) >> 32 from the first word w0 of Philox4x32-10 counter (s, 0, 0, stream)
for snapshot s.  The arithmetic is binary32 round-to-nearest in the written order, so
that the integer decisions match a binary32 implementation exactly.
"""
from __future__ import annotations

import numpy as np

from . import philox4x32_10

f32 = np.float32


def state_at(d0, positions, ts):
    """Positions after ts steps: the snapshot state (positions[t] holds the state after step t)."""
    return np.asarray(d0, f32) if ts == 0 else np.asarray(positions[ts - 1], f32)


def leader(d):
    """LW: the largest position, equal positions: the lower index."""
    best = 0
    for c in range(1, len(d)):
        if d[c] > d[best]:
            best = c
    return best


def underdog(d, gap):
    p1 = leader(d)
    p2 = None
    for c in range(len(d)):
        if c != p1 and (p2 is None or d[c] > d[p2]):
            p2 = c
    if p2 is not None and f32(d[p1] - d[p2]) < f32(gap):
        return p2
    return p1


def linex(d, steps, ts, window, L, prev0):
    """steps[t] = the step sizes of step t; uses rows ts - w .. ts - 1, w = min(window, ts)."""
    n = len(d)
    w = min(window, ts)
    best, pick = None, 0
    for c in range(n):
        if w == 0:
            v = f32(prev0[c])
        else:
            s = f32(0.0)
            for m in range(ts - w, ts):
                s = f32(s + f32(steps[m][c]))
            v = f32(s / f32(w))
        tc = f32(f32(f32(L) - f32(d[c])) / v)
        if best is None or tc < best:
            best, pick = tc, c
    return pick


def zero_intelligence(n, seed, s, stream):
    w0 = int(philox4x32_10([s, 0, 0, stream], [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])[0])
    return (w0 * n) >> 32
