"""Pins of the oracle's Gaussian noise model (Sec. 2.2, Eqs. 2.2-2.6)."""
import numpy as np
from scipy.optimize import minimize_scalar
from scipy.stats import norm


def _problem(seed, n_rot=5, n_pix=9, n_data=4):
    rng = np.random.default_rng(seed)
    W = rng.uniform(0.1, 5.0, size=(n_rot, n_pix))
    w = rng.uniform(0.5, 1.5, size=n_rot)
    w /= w.sum()
    K = rng.poisson(2.0, size=(n_data, n_pix)).astype(float)
    return W, w, K


def test_fluence_is_least_squares_optimum(oracle):
    # Eq. 2.6 minimises sum_i (K_ik / phi - W_ij)^2 over phi (numerical search)
    W, _, K = _problem(30)
    F = oracle.fluence(W, K)
    for j in range(W.shape[0]):
        for k in range(K.shape[0]):
            res = minimize_scalar(lambda t: ((K[k] * t - W[j]) ** 2).sum(), bounds=(0, 10),
                                  method="bounded", options={"xatol": 1e-12})
            assert abs(F[j, k] - res.x) <= 1e-7
    # and is the stated ratio written the other way up: phi = sum K^2 / sum W K
    assert np.isclose(1.0 / F[2, 1], (K[1] ** 2).sum() / (W[2] * K[1]).sum(), rtol=1e-14)


def test_estep_against_normal_pdf(oracle):
    # P(R_j | K_k) = w_j prod_i N(K_ik / phi_jk; W_ij, sigma) / sum over j
    W, w, K = _problem(31)
    sigma = 1.7
    F = oracle.fluence(W, K)
    S = oracle.scores_gauss(W, w, K, sigma)
    P, lse, _ = oracle.estep(S)
    logp = np.array([[np.log(w[j]) + norm.logpdf(K[k] * F[j, k], W[j], sigma).sum()
                      for k in range(K.shape[0])] for j in range(W.shape[0])])
    ref = np.exp(logp - logp.max(0))
    assert np.allclose(P, ref / ref.sum(0), rtol=0, atol=1e-13)
    # lse differs from the normalised density only by the Gaussian constant
    const = W.shape[1] * np.log(np.sqrt(2 * np.pi) * sigma)
    assert np.allclose(lse, np.log(np.exp(logp - logp.max(0)).sum(0)) + logp.max(0) + const,
                       atol=1e-10)


def test_scores_invariant_to_frame_scale(oracle):
    # K -> c K scales phi by c and leaves K / phi, hence Q, unchanged
    W, w, K = _problem(32)
    S1 = oracle.scores_gauss(W, w, K, 0.9)
    S2 = oracle.scores_gauss(W, w, 3.25 * K, 0.9)
    assert np.allclose(S1, S2, rtol=0, atol=1e-11)


def test_scores_bounded_by_prior(oracle):
    # Cauchy-Schwarz: Q_jk <= 0, with equality when K_k is proportional to W_j
    W, w, K = _problem(33)
    K[2] = 1.5 * W[3]
    S = oracle.scores_gauss(W, w, K, 1.1)
    assert np.all(S <= np.log(w)[:, None] + 1e-12)
    assert abs(S[3, 2] - np.log(w[3])) <= 1e-12
    # an empty frame scores -sum W^2 / (2 sigma^2) whatever its fluence
    K[1] = 0.0
    S = oracle.scores_gauss(W, w, K, 1.1)
    assert np.allclose(S[:, 1], -(W ** 2).sum(1) / (2 * 1.1 ** 2) + np.log(w), atol=1e-12)


def test_mstep_recovers_scaled_slices(oracle):
    # frames that are slices times a fluence, with one-hot P: Num / den = the slices
    W, _, _ = _problem(34, n_rot=4, n_pix=11)
    alpha = np.array([0.5, 2.0, 3.0, 1.25, 7.0])
    j_of = np.array([2, 0, 2, 3, 1])
    K = alpha[:, None] * W[j_of]
    P = np.zeros((4, 5))
    P[j_of, np.arange(5)] = 1.0
    Num, den = oracle.mstep_gauss(P, K, oracle.fluence(W, K))
    assert np.allclose(den, [1, 1, 2, 1])
    assert np.allclose(Num / den[:, None], W, rtol=1e-13)
    # a plain P K (no fluence) would give alpha-weighted slices instead
    assert not np.allclose((P @ K) / den[:, None], W, rtol=1e-3)


def test_iteration_keeps_a_constant_model(oracle, small_problem):
    # constant model, frames = fluence x constant: every used slice is the
    # constant, so Eq. 2.12 returns it on every touched voxel; others keep it too
    p = small_problem
    N = p["N"]
    grid = np.full((N, N, N), 2.5)
    K = np.outer(np.array([1.0, 3.0, 0.5, 2.0]), np.full(p["q"].shape[0], 2.5))
    out, lse, L = oracle.iteration_gauss(grid, p["quat"][:200], p["w"][:200] / p["w"][:200].sum(),
                                         p["q"], K, 1.0)
    assert np.allclose(out, 2.5, rtol=1e-12)
    assert np.isfinite(L)


def test_iteration_matches_steps(oracle, small_problem):
    # the fused iteration equals its steps called one by one
    p = small_problem
    quat, w = p["quat"][:150], p["w"][:150] / p["w"][:150].sum()
    K = p["K"][:40]
    out, lse, L, P = oracle.iteration_gauss(p["grid"], quat, w, p["q"], K, 1.3, want_P=True)
    W = oracle.expand(p["grid"], quat, p["q"], 0.0)
    F = oracle.fluence(W, K)
    P2, lse2, L2 = oracle.estep(oracle.scores_gauss(W, w, K, 1.3, F))
    Num, den = oracle.mstep_gauss(P2, K, F)
    out2, _, _ = oracle.compress(p["N"], quat, p["q"], Num, den, p["grid"])
    assert np.allclose(P, P2, atol=1e-15) and np.allclose(lse, lse2) and np.isclose(L, L2)
    assert np.allclose(out, out2, rtol=1e-14)
