"""Pins of the oracle's e-step (Eq. 2.9) and c-step (Eqs. 2.10, 2.12)."""
import numpy as np


def _ball(rng, n, r):
    # n points uniform in a ball of radius r (rotated points stay inside the grid)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * r * rng.random(n)[:, None] ** (1 / 3)


def _grid_points(oracle, quat, q, N):
    R = oracle.quat_to_matrix(quat)
    return np.einsum("jab,ib->jia", R, q) + N / 2


def test_trilinear_reproduces_affine_fields(oracle):
    # trilinear interpolation is exact on affine functions of the grid index
    N = 16
    quat, _ = oracle.quat_generate(2)
    rng = np.random.default_rng(0)
    q = _ball(rng, 50, 6.0)
    a, b = 3.0, np.array([0.25, -0.1, 0.05])
    idx = np.stack(np.meshgrid(*[np.arange(N)] * 3, indexing="ij"), -1)
    grid = a + idx @ b
    W = oracle.expand(grid, quat, q, 1e-30)
    expect = a + _grid_points(oracle, quat, q, N) @ b
    assert np.abs(W - expect).max() < 1e-12


def test_constant_grid_and_grid_points(oracle):
    N = 12
    quat, _ = oracle.quat_generate(1)
    q = _ball(np.random.default_rng(1), 20, 4.0)
    W = oracle.expand(np.full((N, N, N), 2.5), quat, q, 1e-30)
    assert np.allclose(W, 2.5, rtol=0, atol=1e-13)
    # identity rotation, pixels on grid points: W is the voxel value itself
    grid = np.random.default_rng(2).uniform(1, 2, size=(N, N, N))
    qi = np.array([[1.0, -2.0, 3.0], [0.0, 0.0, 0.0], [-5.0, 4.0, -1.0]])
    W = oracle.expand(grid, np.array([[1.0, 0, 0, 0]]), qi, 1e-30)
    ii = (qi + N / 2).astype(int)
    assert np.allclose(W[0], grid[ii[:, 0], ii[:, 1], ii[:, 2]], rtol=0, atol=1e-15)


def test_floor_applies(oracle):
    N = 8
    W = oracle.expand(np.zeros((N, N, N)), np.array([[1.0, 0, 0, 0]]), np.zeros((3, 3)), 1e-7)
    assert np.all(W == 1e-7)


def test_compress_is_adjoint_of_expand(oracle):
    # <e(G), S> = <G, sum_ij f S_ij>: the c-step numerator scatters with exactly
    # the weights the e-step gathers with
    N = 16
    quat, _ = oracle.quat_generate(2)
    rng = np.random.default_rng(3)
    q = _ball(rng, 40, 6.5)
    G = rng.uniform(0.5, 1.5, size=(N, N, N))
    S = rng.standard_normal((quat.shape[0], q.shape[0]))
    W = oracle.expand(G, quat, q, 1e-30)
    _, gnum, _ = oracle.compress(N, quat, q, S, np.ones(quat.shape[0]), G)
    assert abs(np.sum(W * S) - np.sum(G * gnum)) < 1e-9 * np.abs(W * S).sum()


def test_expand_then_compress_constant_returns_constant(oracle):
    N = 16
    quat, _ = oracle.quat_generate(2)
    rng = np.random.default_rng(4)
    q = _ball(rng, 60, 6.5)
    c = 1.75
    G = np.full((N, N, N), c)
    W = oracle.expand(G, quat, q, 1e-30)
    den = rng.uniform(0.2, 2.0, size=quat.shape[0])
    out, gnum, gden = oracle.compress(N, quat, q, W * den[:, None], den, np.zeros_like(G))
    touched = gden > 0
    assert touched.sum() > 100
    assert np.allclose(out[touched], c, rtol=1e-13)
    assert np.all(out[~touched] == 0)  # untouched voxels keep the previous model
    # IDW form (Eq. 2.5 then Eq. 2.10) gives the constant as well
    out2, _, _ = oracle.compress(N, quat, q, W * den[:, None], den, np.zeros_like(G), mode=1)
    assert np.allclose(out2[touched], c, rtol=1e-13)


def test_deferred_equals_idw_for_equal_denominators(oracle):
    N = 16
    quat, _ = oracle.quat_generate(2)
    rng = np.random.default_rng(5)
    q = _ball(rng, 30, 6.5)
    Num = rng.uniform(0, 3, size=(quat.shape[0], q.shape[0]))
    den = np.full(quat.shape[0], 0.7)
    a, _, _ = oracle.compress(N, quat, q, Num, den, np.ones((N, N, N)), mode=0)
    b, _, _ = oracle.compress(N, quat, q, Num, den, np.ones((N, N, N)), mode=1)
    assert np.allclose(a, b, rtol=1e-13)


def test_single_rotation_mean_of_frames(oracle):
    # M_rot = 1 (identity), pixels on grid points: P = 1, so the new model at a
    # pixel's voxel is the mean count of that pixel over the frames
    N = 10
    qi = np.array([[1.0, 2.0, -3.0], [0.0, -1.0, 2.0], [3.0, 3.0, 3.0], [-4.0, 0.0, 1.0]])
    K = np.random.default_rng(6).poisson(3.0, size=(7, 4)).astype(float)
    grid = np.full((N, N, N), 2.0)
    out, lse, L = oracle.iteration(grid, np.array([[1.0, 0, 0, 0]]), np.array([1.0]), qi, K, 1e-12)
    ii = (qi + N / 2).astype(int)
    assert np.allclose(out[ii[:, 0], ii[:, 1], ii[:, 2]], K.mean(0), rtol=1e-13)


def test_round_trip_error_is_second_order(oracle):
    # Expansion followed by compression with unit weights (Eqs. 2.9, 2.12) is a
    # smoothing operator: on a smooth field its error falls with the square of the
    # field's length scale (trilinear interpolation is second order), so doubling
    # a Gaussian blob's width divides it by 4. Speckles of about 2 voxels lose a
    # quarter of their norm, which is where EMC's fixed point sits against the
    # true intensity of the synthetic particles.
    from paper_1409_4256_gb300 import synth
    N = 32
    q = synth.make_detector(N, N, 0.0).q
    quat, _ = oracle.quat_generate(4)
    ax = np.arange(N) - N // 2
    r2 = ax[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2
    inside = r2 <= (N / 2 - 1) ** 2

    def round_trip_error(G):
        W = oracle.expand(G, quat, q, 0.0)
        out, _, _ = oracle.compress(N, quat, q, W, np.ones(quat.shape[0]), G)
        return np.linalg.norm(out[inside] - G[inside]) / np.linalg.norm(G[inside])

    e2 = round_trip_error(np.exp(-r2 / 8.0))    # sigma 2 voxels
    e4 = round_trip_error(np.exp(-r2 / 32.0))   # sigma 4 voxels
    assert 3.6 < e2 / e4 < 4.4
    assert e4 < 0.02
    atoms = synth.make_atoms(50, 8.0)
    speckled = synth.intensity(synth.grid_points(N), atoms, N).reshape(N, N, N)
    assert 0.2 < round_trip_error(speckled) < 0.3
