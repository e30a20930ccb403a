"""Fit of the polynomial g(f) ~ log(1 + f) / f used by the oracle's natural log (test
infrastructure: it writes constants, it computes no part of the method).

Procedure, fully specified so that the constants can be reproduced:
  * interval [sqrt(1/2) - 1, sqrt(2) - 1] (the range of f = m - 1 after the reduction
    x = 2^e m, m in (sqrt(1/2), sqrt(2)]);
  * g(f) = 1 + c1 f + ... + c9 f^9 (the constant term fixed at 1, so log(1 + f) = f g(f) is
    exact at f = 0);
  * 512 Chebyshev nodes of the first kind on the interval;
  * Lawson's algorithm (C. L. Lawson, 1961: iteratively reweighted least squares converging to
    the minimax solution) on the relative error (1 + sum c_j f^j - y) / y with y = log1p(f) / f,
    starting from equal weights, each round multiplying the weights by the absolute errors and
    normalising them; 50 rounds; float64 throughout (numpy's lstsq);
  * each coefficient rounded once to binary32 (round to nearest).

  python -m oracle.fit_log            prints the ten binary32 constants, c0 .. c9, as C hex floats
  python -m oracle.fit_log --check    exits 1 unless oracle/bbe_oracle.c holds exactly these
"""
from __future__ import annotations

import os
import re
import sys

import numpy as np

NODES = 512
ROUNDS = 50
DEGREE = 9


def fit() -> np.ndarray:
    """The ten binary32 coefficients c0 = 1, c1 .. c9."""
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    k = np.arange(NODES)
    f = (lo + hi) / 2 + (hi - lo) / 2 * np.cos(np.pi * (k + 0.5) / NODES)
    y = np.log1p(f) / f
    A = np.stack([f ** j for j in range(1, DEGREE + 1)], axis=1)
    w = np.full(NODES, 1.0 / NODES)
    for _ in range(ROUNDS + 1):
        s = np.sqrt(w) / y
        c, *_ = np.linalg.lstsq(A * s[:, None], (y - 1.0) * s, rcond=None)
        err = np.abs((1.0 + A @ c - y) / y)
        w = w * err
        w = w / w.sum()
    return np.concatenate([[1.0], c]).astype(np.float32)


def c_hex(x: np.float32) -> str:
    """A binary32 value as a C hex-float literal with six hex digits of fraction."""
    v = float(x)
    if v == 0.0:
        return "0x0p+0f"
    sign = "-" if v < 0 else ""
    m, e = np.frexp(abs(v))                  # v = m 2^e, m in [0.5, 1)
    frac = int(round((m * 2.0 - 1.0) * (1 << 24)))  # 23 fraction bits, shifted left by one
    return f"{sign}0x1.{frac:06x}p{e - 1:+d}f"


def oracle_constants() -> np.ndarray:
    src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bbe_oracle.c")).read()
    body = re.search(r"static const float G\[10\] = \{([^}]*)\};", src).group(1)
    vals = [float.fromhex(t.strip().rstrip("f")) for t in body.split(",") if t.strip()]
    return np.array(vals, np.float32)


def main(argv) -> int:
    g = fit()
    if "--check" in argv:
        ok = np.array_equal(oracle_constants().view(np.uint32), g.view(np.uint32))
        print("oracle constants match the fit" if ok else "oracle constants differ from the fit")
        return 0 if ok else 1
    print(", ".join(c_hex(x) for x in g))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
