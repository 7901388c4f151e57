"""Distances between distributions and sampling from them.
TEST INFRASTRUCTURE ONLY.

chi_square is the chi^2 loss of Eq. 16 (Sec. 5.2), with which the paper
compares an execution's output distribution a against the ground truth b:

    chi^2 = sum_i (a_i - b_i)^2 / (a_i + b_i).

The paper does not say what a term with a_i + b_i = 0 is; read here as 0 (both
distributions give the outcome no weight, so it contributes nothing).
total_variation is (1/2) sum_i |a_i - b_i|, reported beside it.

sample draws outcomes from a reconstructed distribution by inverse transform:
weights w_i = max(p_i, 0) (a reconstructed quasi-probability can be slightly
negative from rounding; negative entries are given no weight), cumulative
sums C_x = sum_{i <= x} w_i in order, and for each uniform u in [0, 1) the
smallest x with C_x > u * C_last.  The uniforms are inputs, so both sides
draw the same outcomes.  When no outcome carries weight (C_last = 0) there is
nothing to draw; every draw is then -1.
"""
from __future__ import annotations

import numpy as np


def chi_square(a, b) -> float:
    """Eq. 16 term by term in FP64; a term with a_i + b_i = 0 is 0."""
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    total = 0.0
    num = (a - b) ** 2
    den = a + b
    for n_i, d_i in zip(num, den):
        if d_i != 0.0:
            total += n_i / d_i
    return float(total)


def total_variation(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(0.5 * np.abs(a - b).sum())


def cumulative(p) -> np.ndarray:
    """C_x = sum_{i <= x} max(p_i, 0), summed in index order."""
    w = np.maximum(np.asarray(p, dtype=np.float64).reshape(-1), 0.0)
    return np.cumsum(w)


def sample(p, u) -> np.ndarray:
    """Outcome index for each uniform u: the smallest x with C_x > u * C_last."""
    C = cumulative(p)
    if not C[-1] > 0.0:
        return np.full(np.shape(u), -1, dtype=np.int64)
    t = np.asarray(u, dtype=np.float64) * C[-1]
    x = np.searchsorted(C, t, side="right")
    return np.minimum(x, len(C) - 1).astype(np.int64)
