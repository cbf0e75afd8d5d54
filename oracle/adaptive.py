"""FP64 oracle of adaptive EMC (Sec. 3.4, Eq. 3.1).

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU legs); the GPU
library never uses it.

The schedule: iterate Algorithm 2.1 at the 600-cell subdivision d (Eq. 2.7);
after iteration n, if the log-likelihood changed by no more than 1% of its
magnitude, |L^n - L^{n-1}| <= 0.01 |L^n|, continue at d + 1 (up to d_max).
L^n is read as the full Poisson log-likelihood of all frames under the mixture
over sampled rotations, sum_k log sum_j w_j prod_i Poisson(K_ik; W_ij): the
E-step's sum_k lse_k minus the data constant sum_ik log K_ik!. The comparison
only starts once two iterations have run at the current d.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle


def log_factorial_constant(K) -> float:
    """sum_ik log(K_ik!) via lgamma, one term per distinct count value."""
    vals, counts = np.unique(np.asarray(K, dtype=np.int64), return_counts=True)
    return float(sum(c * math.lgamma(v + 1.0) for v, c in zip(vals, counts)))


def log_likelihood(lse_sum: float, K) -> float:
    """Full Poisson log-likelihood from the E-step's sum_k lse_k (Eq. 2.4)."""
    return lse_sum - log_factorial_constant(K)


def should_refine(L_now: float, L_prev, threshold: float = 0.01) -> bool:
    """Eq. 3.1: move to a finer rotation sampling when the change is small."""
    if L_prev is None:
        return False
    return abs(L_now - L_prev) <= threshold * abs(L_now)


def run(grid, q, K, d0: int, d_max: int, iterations: int, w_floor: float,
        threshold: float = 0.01, mode: int = 0):
    """Adaptive EMC from `grid`: returns (grid, [(d, n_rot, L), ...])."""
    grid = np.asarray(grid, dtype=np.float64)
    d, L_prev, hist = d0, None, []
    for _ in range(iterations):
        quat, w = oracle.quat_generate(d)
        grid, _, tot = oracle.iteration(grid, quat, w, q, K, w_floor, mode)
        L = log_likelihood(tot, K)
        hist.append((d, quat.shape[0], L))
        if should_refine(L, L_prev, threshold) and d < d_max:
            d, L_prev = d + 1, None
        else:
            L_prev = L
    return grid, hist
