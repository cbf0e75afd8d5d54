"""Pins of the oracle's E-step (Eq. 2.4, Poisson model) and M-step (Eq. 2.11)."""
import numpy as np
import pytest
from scipy.special import gammaln
from scipy.stats import poisson


def test_estep_against_poisson_pmf(oracle):
    # brute force: P(R_j | K_k) = w_j prod_i pmf(K_ik; W_ij) / sum_j' (...)
    rng = np.random.default_rng(10)
    n_rot, n_pix, n_data = 5, 7, 3
    W = rng.uniform(0.2, 4.0, size=(n_rot, n_pix))
    w = rng.uniform(0.5, 1.5, size=n_rot)
    w /= w.sum()
    K = rng.poisson(1.5, size=(n_data, n_pix)).astype(float)
    S = oracle.scores(W, w, K)
    P, lse, tot = oracle.estep(S)
    lik = np.array([[w[j] * np.prod(poisson.pmf(K[k], W[j])) for k in range(n_data)]
                    for j in range(n_rot)])
    assert np.allclose(P, lik / lik.sum(0), rtol=1e-11, atol=0)
    # lse_k = log sum_j w_j prod_i pmf + sum_i log K_ik! (the dropped constant)
    expect = np.log(lik.sum(0)) + gammaln(K + 1).sum(1)
    assert np.allclose(lse, expect, rtol=0, atol=1e-10)
    assert np.isclose(tot, expect.sum(), rtol=0, atol=1e-9)


def test_scores_transposition_sensitive(oracle):
    # asymmetric sizes and one hand-checked element
    W = np.array([[1.0, 2.0, 3.0], [0.5, 0.25, 4.0]])
    w = np.array([0.25, 0.75])
    K = np.array([[1.0, 0.0, 2.0]])
    S = oracle.scores(W, w, K)
    assert S.shape == (2, 1)
    assert np.isclose(S[1, 0], 1 * np.log(0.5) + 2 * np.log(4.0) - (0.5 + 0.25 + 4.0) + np.log(0.75))


def test_responsibilities_sum_to_one_and_shift_invariant(oracle):
    rng = np.random.default_rng(11)
    S = rng.normal(0, 30, size=(40, 9)) + 5000.0  # naive exp would overflow
    P, lse, _ = oracle.estep(S)
    assert np.allclose(P.sum(0), 1.0, atol=1e-13)
    P2, lse2, _ = oracle.estep(S - 4000.0)
    assert np.allclose(P, P2, atol=1e-14) and np.allclose(lse - lse2, 4000.0, atol=1e-9)


def test_single_rotation_gives_certainty(oracle):
    rng = np.random.default_rng(12)
    S = rng.normal(size=(1, 6))
    P, lse, _ = oracle.estep(S)
    assert np.all(P == 1.0) and np.allclose(lse, S[0])


def test_mstep_matches_matrix_product(oracle):
    rng = np.random.default_rng(13)
    P = rng.uniform(size=(6, 11))
    K = rng.poisson(2.0, size=(11, 5)).astype(float)
    Num, den = oracle.mstep(P, K)
    assert np.allclose(Num, P @ K, rtol=1e-13) and np.allclose(den, P.sum(1), rtol=1e-13)


def test_em_without_compression_never_decreases_likelihood(oracle):
    # EM theorem: with W_ij free per (i, j), the M-step W'_ij = Num_ij / den_j
    # is the Poisson maximiser given P, so the observed-data likelihood
    # sum_k lse_k cannot decrease. A wrong M-step (dropped den, wrong index)
    # breaks this.
    rng = np.random.default_rng(14)
    n_rot, n_pix, n_data = 12, 25, 40
    truth = rng.gamma(2.0, 1.0, size=(n_rot, n_pix))
    lab = rng.integers(0, n_rot, size=n_data)
    K = rng.poisson(truth[lab]).astype(float)
    w = np.full(n_rot, 1.0 / n_rot)
    W = rng.gamma(2.0, 1.0, size=(n_rot, n_pix))
    prev = -np.inf
    for _ in range(8):
        P, lse, L = oracle.estep(oracle.scores(W, w, K))
        assert L >= prev - 1e-9
        prev = L
        Num, den = oracle.mstep(P, K)
        W = np.maximum(Num / den[:, None], 1e-12)


def test_noiseless_frames_recover_their_rotation(oracle):
    # frames sliced (without noise) from a known model at sampled rotations:
    # the best-scoring rotation is the one they were sliced at
    from paper_1409_4256_gb300 import synth
    quat, w = oracle.quat_generate(3)
    sel = np.random.default_rng(15).choice(quat.shape[0], size=12, replace=False)
    Rt = oracle.quat_to_matrix(quat[sel])
    ds = synth.make_dataset(32, 32, 12, 20.0, radius=8.0, rot_true=Rt, noiseless=True)
    W = oracle.expand(ds.model_true, quat, ds.q, 1e-10 * ds.model_true.mean())
    S = oracle.scores(W, w, ds.K)
    assert np.all(np.argmax(S, axis=0) == sel)
