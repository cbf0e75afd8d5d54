"""Adaptive EMC (Sec. 3.4, Eq. 3.1): start from a coarse rotation sampling and
refine it as the likelihood stops improving.

The paper increases the subdivision d of the 600-cell sampling (Eq. 2.7) by
one whenever |L^n - L^{n-1}| <= 0.01 |L^n|, L^n being the log-likelihood at
iteration n. Reading: L^n is the full Poisson log-likelihood of the frames,
sum_k lse_k - sum_ik log K_ik! (the second term is a constant of the data but
fixes the scale the relative criterion compares against).

Every iteration runs in libemc (emc_iteration); this driver only keeps the
schedule, the model grid between iterations and a context per sampling level.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import emc


def log_factorial_sum(K: np.ndarray) -> float:
    """sum_ik log K_ik! of integer counts (exact table up to the largest count)."""
    K = np.asarray(K)
    kmax = int(K.max()) if K.size else 0
    table = np.concatenate([[0.0], np.cumsum(np.log(np.arange(1, kmax + 1, dtype=np.float64)))])
    counts = np.bincount(K.ravel(), minlength=kmax + 1)
    return float(counts @ table)


def refine(L_now: float, L_prev: float | None, threshold: float = 0.01) -> bool:
    """Eq. 3.1: refine when the likelihood changed by at most threshold |L^n|."""
    return L_prev is not None and abs(L_now - L_prev) <= threshold * abs(L_now)


@dataclasses.dataclass
class Step:
    iteration: int
    d: int
    n_rot: int
    loglik: float
    ms: float


def run(N: int, q: np.ndarray, K, grid, d0: int, d_max: int, iterations: int, *,
        threshold: float = 0.01, precision="bf16_split", w_floor: float = 1e-10,
        store_scores: bool = True, device="cuda", K_host: np.ndarray | None = None,
        callback=None, stream=None):
    """Adaptive EMC on frames K (device int32 [n_data, n_pix]) from `grid`
    (device float32 [N, N, N]). Returns (grid, [Step, ...]).

    callback(step, grid_in, grid_out), if given, runs after every iteration
    (device tensors; grid_in is overwritten two iterations later). Step.ms is
    the iteration's device time (CUDA events inside emc_iteration)."""
    import torch
    n_data = K.shape[0]
    const = log_factorial_sum(K_host if K_host is not None else K.cpu().numpy())
    d = d0
    ctx = None
    hist: list[Step] = []
    L_prev = None
    cur = grid.clone()  # the caller's grid is left as it is
    nxt = torch.empty_like(cur)
    if stream is not None:
        cur.record_stream(stream)
        nxt.record_stream(stream)
        stream.wait_stream(torch.cuda.current_stream(grid.device))
    for it in range(iterations):
        if ctx is None:
            quat, w = emc.quat_generate(d)
            ctx = emc.Context(N, q, quat, w, n_data, precision=precision, w_floor=w_floor,
                              store_scores=store_scores, device=device, stream=stream)
            ctx.set_frames(K, stream=stream)
        _, st = ctx.iteration(cur, nxt, stream=stream)
        if st["device_status"] != 0:
            raise emc.EmcError(f"device status {st['device_status']} at iteration {it}")
        L = st["loglik"] - const
        hist.append(Step(it, d, ctx.cfg.n_rot, L, st["ms_total"]))
        if callback is not None:
            callback(hist[-1], cur, nxt)
        cur, nxt = nxt, cur
        if refine(L, L_prev, threshold) and d < d_max:
            d += 1
            ctx = None  # the next iteration samples rotations at the finer level
            L_prev = None
        else:
            L_prev = L
    return cur, hist
