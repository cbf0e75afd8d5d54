"""ctypes front end of the FP64 CPU oracle (emc_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use it; the GPU library never does. Functions mirror the C entry
points one to one and take/return float64 numpy arrays. See emc_oracle.c for
the paper passage each one follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "emc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2, IEEE semantics, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.oracle_quat_generate.restype = ctypes.c_long
            L.oracle_quat_generate.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_long]
            L.oracle_600cell_counts.restype = ctypes.c_long
            L.oracle_600cell_counts.argtypes = [ctypes.POINTER(ctypes.c_long)] * 2
            L.oracle_quat_to_matrix.argtypes = [_dp, _dp]
            L.oracle_expand.argtypes = [ctypes.c_int, _dp, ctypes.c_long, _dp, ctypes.c_long, _dp,
                                        ctypes.c_double, _dp]
            L.oracle_scores.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp]
            L.oracle_estep.restype = ctypes.c_double
            L.oracle_estep.argtypes = [ctypes.c_long, ctypes.c_long, _dp, _dp, _dp]
            L.oracle_mstep.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_long, _dp, _dp, _dp, _dp]
            L.oracle_compress.argtypes = [ctypes.c_int, ctypes.c_long, _dp, ctypes.c_long, _dp, _dp,
                                          _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
            L.oracle_iteration.restype = ctypes.c_double
            L.oracle_iteration.argtypes = [ctypes.c_int, _dp, ctypes.c_long, _dp, _dp, ctypes.c_long,
                                           _dp, ctypes.c_long, _dp, ctypes.c_double, ctypes.c_int,
                                           _dp, _dp, _dp]
            L.oracle_fluence.argtypes = [ctypes.c_long] * 3 + [_dp] * 3
            L.oracle_scores_gauss.argtypes = [ctypes.c_long] * 3 + [_dp] * 3 + [ctypes.c_double,
                                                                                _dp, _dp]
            L.oracle_mstep_gauss.argtypes = [ctypes.c_long] * 3 + [_dp] * 5
            L.oracle_iteration_gauss.restype = ctypes.c_double
            L.oracle_iteration_gauss.argtypes = [ctypes.c_int, _dp, ctypes.c_long, _dp, _dp,
                                                 ctypes.c_long, _dp, ctypes.c_long, _dp,
                                                 ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            L.oracle_fluence_poisson.argtypes = [ctypes.c_long] * 3 + [_dp] * 3
            L.oracle_scores_poisson_fluence.argtypes = [ctypes.c_long] * 3 + [_dp] * 5
            L.oracle_iteration_poisson_fluence.restype = ctypes.c_double
            L.oracle_iteration_poisson_fluence.argtypes = [ctypes.c_int, _dp, ctypes.c_long, _dp,
                                                           _dp, ctypes.c_long, _dp, ctypes.c_long,
                                                           _dp, ctypes.c_double, ctypes.c_int,
                                                           _dp, _dp, _dp]
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(_dp)


def num_threads() -> int:
    return lib().oracle_num_threads()


def cell_counts() -> tuple[int, int, int]:
    """(vertices, edges, cells) of the 600-cell as the oracle constructs it."""
    nv, ne = ctypes.c_long(), ctypes.c_long()
    nc = lib().oracle_600cell_counts(ctypes.byref(nv), ctypes.byref(ne))
    return nv.value, ne.value, nc


def quat_generate(n: int, uniform: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 2.7 sampling: (quat[M_rot, 4] (w,x,y,z), weight[M_rot] summing to 1)."""
    L = lib()
    m = L.oracle_quat_generate(n, int(uniform), None, None, 0)
    if m < 0:
        raise RuntimeError(f"oracle_quat_generate failed ({m})")
    quat = np.empty((m, 4))
    w = np.empty(m)
    r = L.oracle_quat_generate(n, int(uniform), _p(quat), _p(w), m)
    if r != m:
        raise RuntimeError(f"oracle_quat_generate failed ({r})")
    return quat, w


def quat_to_matrix(quat) -> np.ndarray:
    quat = _f64(np.atleast_2d(quat))
    out = np.empty((quat.shape[0], 3, 3))
    for j in range(quat.shape[0]):
        lib().oracle_quat_to_matrix(_p(quat[j]), _p(out[j]))
    return out


def expand(grid, quat, q, w_floor: float) -> np.ndarray:
    """Eq. 2.9 with floor: W[n_rot, n_pix]."""
    grid, quat, q = _f64(grid), _f64(quat), _f64(q)
    N = grid.shape[0]
    W = np.empty((quat.shape[0], q.shape[0]))
    lib().oracle_expand(N, _p(grid), quat.shape[0], _p(quat), q.shape[0], _p(q), w_floor, _p(W))
    return W


def scores(W, weight, K) -> np.ndarray:
    """Poisson S_jk = sum_i K_ik log W_ij - W_ij + log w_j: [n_rot, n_data]."""
    W, weight, K = _f64(W), _f64(weight), _f64(K)
    S = np.empty((W.shape[0], K.shape[0]))
    lib().oracle_scores(W.shape[0], W.shape[1], K.shape[0], _p(W), _p(weight), _p(K), _p(S))
    return S


def estep(S) -> tuple[np.ndarray, np.ndarray, float]:
    """Eq. 2.4: (P[n_rot, n_data], lse[n_data], sum_k lse_k)."""
    S = _f64(S)
    P = np.empty_like(S)
    lse = np.empty(S.shape[1])
    tot = lib().oracle_estep(S.shape[0], S.shape[1], _p(S), _p(P), _p(lse))
    return P, lse, tot


def mstep(P, K) -> tuple[np.ndarray, np.ndarray]:
    """Eq. 2.11: (Num[n_rot, n_pix], den[n_rot])."""
    P, K = _f64(P), _f64(K)
    Num = np.empty((P.shape[0], K.shape[1]))
    den = np.empty(P.shape[0])
    lib().oracle_mstep(P.shape[0], K.shape[1], P.shape[1], _p(P), _p(K), _p(Num), _p(den))
    return Num, den


def compress(N: int, quat, q, Num, den, grid_prev, mode: int = 0):
    """Eq. 2.12 (mode 0) or Eq. 2.5 + 2.10 (mode 1): (grid_out, g_num, g_den)."""
    quat, q, Num, den, grid_prev = _f64(quat), _f64(q), _f64(Num), _f64(den), _f64(grid_prev)
    gn = np.empty((N, N, N))
    gd = np.empty((N, N, N))
    out = np.empty((N, N, N))
    lib().oracle_compress(N, quat.shape[0], _p(quat), q.shape[0], _p(q), _p(Num), _p(den), mode,
                          _p(grid_prev), _p(gn), _p(gd), _p(out))
    return out, gn, gd


def iteration(grid, quat, weight, q, K, w_floor: float, mode: int = 0, want_P: bool = False):
    """Algorithm 2.1, one pass: (grid_out, lse, loglik[, P])."""
    grid, quat, weight, q, K = _f64(grid), _f64(quat), _f64(weight), _f64(q), _f64(K)
    N = grid.shape[0]
    out = np.empty_like(grid)
    lse = np.empty(K.shape[0])
    P = np.empty((quat.shape[0], K.shape[0])) if want_P else None
    L = lib().oracle_iteration(N, _p(grid), quat.shape[0], _p(quat), _p(weight), q.shape[0], _p(q),
                               K.shape[0], _p(K), w_floor, mode, _p(out), _p(P), _p(lse))
    if want_P:
        return out, lse, L, P
    return out, lse, L


# ----------------------------------------------------------------------------
# Gaussian noise model (Eqs. 2.2-2.3, 2.5-2.6)
# ----------------------------------------------------------------------------

def fluence(W, K) -> np.ndarray:
    """1/phi_jk of Eq. 2.6 (0 for an empty frame): [n_rot, n_data]."""
    W, K = _f64(W), _f64(K)
    F = np.empty((W.shape[0], K.shape[0]))
    lib().oracle_fluence(W.shape[0], W.shape[1], K.shape[0], _p(W), _p(K), _p(F))
    return F


def scores_gauss(W, weight, K, sigma: float, inv_phi=None) -> np.ndarray:
    """S_jk = -sum_i (K_ik / phi_jk - W_ij)^2 / (2 sigma^2) + log w_j."""
    W, weight, K = _f64(W), _f64(weight), _f64(K)
    F = fluence(W, K) if inv_phi is None else _f64(inv_phi)
    S = np.empty((W.shape[0], K.shape[0]))
    lib().oracle_scores_gauss(W.shape[0], W.shape[1], K.shape[0], _p(W), _p(weight), _p(K),
                              float(sigma), _p(F), _p(S))
    return S


def mstep_gauss(P, K, inv_phi) -> tuple[np.ndarray, np.ndarray]:
    """(Num_ij = sum_k P_jk K_ik / phi_jk, den_j = sum_k P_jk)."""
    P, K, F = _f64(P), _f64(K), _f64(inv_phi)
    Num = np.empty((P.shape[0], K.shape[1]))
    den = np.empty(P.shape[0])
    lib().oracle_mstep_gauss(P.shape[0], K.shape[1], P.shape[1], _p(P), _p(K), _p(F), _p(Num),
                             _p(den))
    return Num, den


def iteration_gauss(grid, quat, weight, q, K, sigma: float, mode: int = 0,
                    want_P: bool = False):
    """Algorithm 2.1 under the Gaussian model: (grid_out, lse, sum lse[, P])."""
    grid, quat, weight, q, K = _f64(grid), _f64(quat), _f64(weight), _f64(q), _f64(K)
    N = grid.shape[0]
    out = np.empty_like(grid)
    lse = np.empty(K.shape[0])
    P = np.empty((quat.shape[0], K.shape[0])) if want_P else None
    L = lib().oracle_iteration_gauss(N, _p(grid), quat.shape[0], _p(quat), _p(weight),
                                     q.shape[0], _p(q), K.shape[0], _p(K), float(sigma), mode,
                                     _p(out), _p(P), _p(lse))
    if want_P:
        return out, lse, L, P
    return out, lse, L


# ----------------------------------------------------------------------------
# Poisson model with per-(j,k) fluence (maximum-likelihood scale)
# ----------------------------------------------------------------------------

def fluence_poisson(W, K) -> np.ndarray:
    """1/phi_jk = sum_i W_ij / N_k (0 for an empty frame): [n_rot, n_data]."""
    W, K = _f64(W), _f64(K)
    F = np.empty((W.shape[0], K.shape[0]))
    lib().oracle_fluence_poisson(W.shape[0], W.shape[1], K.shape[0], _p(W), _p(K), _p(F))
    return F


def scores_poisson_fluence(W, weight, K, inv_phi=None) -> np.ndarray:
    """S_jk = sum_i (K log(phi W) - phi W) + log w_j - (N_k log N_k - N_k)."""
    W, weight, K = _f64(W), _f64(weight), _f64(K)
    F = fluence_poisson(W, K) if inv_phi is None else _f64(inv_phi)
    S = np.empty((W.shape[0], K.shape[0]))
    lib().oracle_scores_poisson_fluence(W.shape[0], W.shape[1], K.shape[0], _p(W), _p(weight),
                                        _p(K), _p(F), _p(S))
    return S


def iteration_poisson_fluence(grid, quat, weight, q, K, w_floor: float, mode: int = 0,
                              want_P: bool = False):
    """Algorithm 2.1 under the Poisson-fluence model: (grid_out, lse, sum lse[, P])."""
    grid, quat, weight, q, K = _f64(grid), _f64(quat), _f64(weight), _f64(q), _f64(K)
    N = grid.shape[0]
    out = np.empty_like(grid)
    lse = np.empty(K.shape[0])
    P = np.empty((quat.shape[0], K.shape[0])) if want_P else None
    L = lib().oracle_iteration_poisson_fluence(N, _p(grid), quat.shape[0], _p(quat), _p(weight),
                                               q.shape[0], _p(q), K.shape[0], _p(K), w_floor,
                                               mode, _p(out), _p(P), _p(lse))
    if want_P:
        return out, lse, L, P
    return out, lse, L
