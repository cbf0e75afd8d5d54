"""Pins of the oracle's Poisson model with per-(j,k) fluence."""
import numpy as np
from scipy.optimize import minimize_scalar
from scipy.special import gammaln
from scipy.stats import poisson


def _problem(seed, n_rot=5, n_pix=9, n_data=4):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.1, 5.0, size=(n_rot, n_pix))
    w = rng.uniform(0.5, 1.5, size=n_rot)
    w /= w.sum()
    K = rng.poisson(2.0, size=(n_data, n_pix)).astype(float)
    return W, w, K


def test_fluence_is_the_poisson_mle(oracle):
    W, _, K = _problem(60)
    F = oracle.fluence_poisson(W, K)
    for j in range(W.shape[0]):
        for k in range(K.shape[0]):
            res = minimize_scalar(lambda phi: -poisson.logpmf(K[k], phi * W[j]).sum(),
                                  bounds=(1e-3, 20), method="bounded", options={"xatol": 1e-10})
            assert abs(1.0 / F[j, k] - res.x) <= 1e-6 * res.x


def test_scores_against_poisson_pmf(oracle):
    # S - sum log K! + (N log N - N) = sum_i log pmf(K_ik; phi_jk W_ij) + log w_j
    W, w, K = _problem(61)
    F = oracle.fluence_poisson(W, K)
    S = oracle.scores_poisson_fluence(W, w, K, F)
    N = K.sum(1)
    for j in range(W.shape[0]):
        for k in range(K.shape[0]):
            want = poisson.logpmf(K[k], W[j] / F[j, k]).sum() + np.log(w[j])
            got = S[j, k] - gammaln(K[k] + 1).sum() + (N[k] * np.log(N[k]) - N[k])
            assert abs(got - want) <= 1e-10 * abs(want)


def test_scale_free_frames_and_empty_frames(oracle):
    # K = c W_j exactly: the fitted scale is c and the slice fits as well as any
    W, w, K = _problem(62)
    K[1] = 2.5 * W[3]
    F = oracle.fluence_poisson(W, K)
    assert np.isclose(1.0 / F[3, 1], 2.5, rtol=1e-13)
    K[2] = 0.0
    S = oracle.scores_poisson_fluence(W, w, K)
    assert np.allclose(S[:, 2], np.log(w), atol=1e-14)  # phi = 0: nothing observed


def test_iteration_keeps_a_constant_model(oracle, small_problem):
    # frames = fluence x constant model: every used slice returns the constant
    p = small_problem
    N = p["N"]
    grid = np.full((N, N, N), 2.0)
    K = np.outer(np.array([1.0, 3.0, 0.5]), np.full(p["q"].shape[0], 2.0))
    out, _, L = oracle.iteration_poisson_fluence(grid, p["quat"][:200],
                                                 p["w"][:200] / p["w"][:200].sum(), p["q"], K,
                                                 1e-10)
    assert np.allclose(out, 2.0, rtol=1e-12) and np.isfinite(L)
