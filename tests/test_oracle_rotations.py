"""Pins of the oracle's rotation sampling (Eq. 2.7) against closed forms and
the geometry of SO(3); none of them re-runs the oracle's own formula."""
import os

import numpy as np
import pytest


def test_600cell_incidence(oracle):
    # the 600-cell: 120 vertices, 720 edges, 600 tetrahedral cells
    assert oracle.cell_counts() == (120, 720, 600)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_count_closed_form(oracle, n):
    quat, w = oracle.quat_generate(n)
    assert quat.shape == (10 * (5 * n ** 3 + n), 4)


def printed_counts():
    """(d, M_rot) pairs printed with Eq. 2.7 (tests/golden)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "eq2_7_rotation_counts.txt")
    with open(path) as f:
        rows = [line.split() for line in f if line.strip() and not line.startswith("#")]
    return [(int(d), int(m)) for d, m in rows]


def test_counts_printed_in_paper(oracle):
    # every count printed with Eq. 2.7, generated by the oracle's exact
    # subdivision of the 600-cell (its rotations, not its formula)
    pairs = printed_counts()
    assert [d for d, _ in pairs] == [5, 6, 8, 10, 12]
    for d, m in pairs:
        assert oracle.quat_generate(d)[0].shape[0] == m


def test_incidence_count_by_faces(oracle):
    # distinct lattice points before q ~ -q: vertices + edge interiors +
    # face interiors + cell interiors of the subdivided 600-cell
    from math import comb
    for n in (2, 3, 4):
        pts = 120 + 720 * (n - 1) + 1200 * comb(n - 1, 2) + 600 * comb(n - 1, 3)
        assert oracle.quat_generate(n)[0].shape[0] == pts // 2


def test_unit_canonical_distinct(oracle):
    quat, w = oracle.quat_generate(4)
    assert np.allclose(np.linalg.norm(quat, axis=1), 1.0, atol=1e-14)
    first = quat[np.arange(len(quat)), np.argmax(np.abs(quat) > 1e-12, axis=1)]
    assert np.all(first > 0)
    # no two rotations equal (up to sign): |<q, q'>| < 1 - margin
    G = np.abs(quat @ quat.T)
    np.fill_diagonal(G, 0)
    assert G.max() < 1 - 1e-6


def test_weights_normalised_positive(oracle):
    _, w = oracle.quat_generate(5)
    assert np.all(w > 0) and abs(w.sum() - 1) < 1e-12
    _, wu = oracle.quat_generate(5, uniform=True)
    assert np.allclose(wu, 1.0 / len(wu))


def test_low_moments_exact(oracle):
    # the sampling inherits the 600-cell's symmetry: E[q q^T] = I/4 and
    # E[R] = 0 exactly (to rounding) for any n
    for n in (2, 4):
        quat, w = oracle.quat_generate(n)
        M = (quat * w[:, None]).T @ quat
        ER = np.einsum("j,jab->ab", w, oracle.quat_to_matrix(quat))
        assert np.abs(M - np.eye(4) / 4).max() < 1e-12 and np.abs(ER).max() < 1e-12


def _haar_mean_peaked(kappa):
    # E[exp(kappa (q.u)^2)] for q uniform on S^3: q.u has density
    # (2/pi) sqrt(1 - x^2) on [-1, 1]; evaluated by 1-D quadrature
    from scipy.integrate import quad
    return quad(lambda x: 2 / np.pi * np.sqrt(1 - x * x) * np.exp(kappa * x * x), -1, 1,
                epsabs=1e-14)[0]


@pytest.mark.parametrize("kappa", [10.0, 30.0])
def test_weights_integrate_haar_measure(oracle, kappa):
    # The prior weights must turn the sampling into a quadrature of the uniform
    # measure: the error on a sharply peaked function falls with n, while equal
    # weights keep a bias (the projected lattice crowds near the cell vertices).
    rng = np.random.default_rng(3)
    u = rng.standard_normal(4)
    u /= np.linalg.norm(u)
    exact = _haar_mean_peaked(kappa)
    err_w, err_u = [], []
    for n in (3, 4, 6, 8):
        q, w = oracle.quat_generate(n)
        f = np.exp(kappa * (q @ u) ** 2)
        err_w.append(abs(w @ f / exact - 1))
        err_u.append(abs(f.mean() / exact - 1))
    assert all(a > b for a, b in zip(err_w, err_w[1:]))
    assert err_w[-1] < err_u[-1] / 20
    assert err_w[-1] < 1e-4


def test_rotation_matrices(oracle):
    quat, _ = oracle.quat_generate(2)
    R = oracle.quat_to_matrix(quat)
    I = np.einsum("jab,jcb->jac", R, R)
    assert np.allclose(I, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-13)
    # q and -q give the same rotation
    assert np.allclose(oracle.quat_to_matrix(-quat), R, atol=1e-15)
    # textbook special case: rotation by angle a about z
    a = 0.3
    q = np.array([np.cos(a / 2), 0, 0, np.sin(a / 2)])
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    assert np.allclose(oracle.quat_to_matrix(q)[0], Rz, atol=1e-15)
    # composition: R(q1 q2) = R(q1) R(q2) for the Hamilton product
    def hprod(p, r):
        w1, x1, y1, z1 = p
        w2, x2, y2, z2 = r
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    p, r = quat[5], quat[17]
    assert np.allclose(oracle.quat_to_matrix(hprod(p, r))[0],
                       oracle.quat_to_matrix(p)[0] @ oracle.quat_to_matrix(r)[0], atol=1e-14)


def test_covering_radius_shrinks(oracle):
    # every Haar-random rotation has a sampled neighbour, closer for larger n
    from paper_1409_4256_gb300 import synth
    Rt = synth.random_rotations(200, seed=7)
    prev = None
    for n in (2, 4, 6):
        quat, _ = oracle.quat_generate(n)
        R = oracle.quat_to_matrix(quat)
        cos = (np.einsum("kab,jab->kj", Rt, R) - 1) / 2
        ang = np.arccos(np.clip(cos.max(1), -1, 1))
        if prev is not None:
            assert ang.max() < prev
        prev = ang.max()
    assert prev < 0.2
