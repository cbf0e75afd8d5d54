"""Pins of the learned-proposal oracle (oracle/learned.py) against finite
differences, closed forms and the (already pinned) dense oracle."""
import numpy as np
import pytest

from oracle import learned as ol


def _tiny_params(rng, dims):
    ps = []
    for a, b in zip(dims[:-1], dims[1:]):
        ps.append(rng.normal(0, 1 / np.sqrt(a), size=(a, b)))
        ps.append(rng.normal(0, 0.1, size=b))
    return ps


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(0)
    params = _tiny_params(rng, [6, 5, 5, 5, 7])
    X = rng.normal(size=(4, 6))
    T = rng.random((4, 7))
    T /= T.sum(axis=1, keepdims=True)
    loss, grads = ol.mlp_loss_grads(params, X, T)
    h = 1e-6
    for i, p in enumerate(params):
        num = np.zeros_like(p)
        for idx in np.ndindex(p.shape):
            old = p[idx]
            p[idx] = old + h
            lp = ol.soft_ce_loss(ol.mlp_forward(params, X)[0], T)
            p[idx] = old - h
            lm = ol.soft_ce_loss(ol.mlp_forward(params, X)[0], T)
            p[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(grads[i], num, rtol=1e-6, atol=1e-9), i


def test_gelu_closed_forms():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    from math import erf, sqrt
    assert np.allclose(ol.gelu(x), [0.5 * v * (1 + erf(v / sqrt(2))) for v in x], rtol=1e-14)
    h = 1e-6
    assert np.allclose(ol.gelu_grad(x), (ol.gelu(x + h) - ol.gelu(x - h)) / (2 * h), rtol=1e-7)


def test_adam_first_step_is_signed_lr():
    # bias correction makes the first step -lr * g / (|g| + eps)
    p = [np.array([1.0, -2.0, 3.0])]
    g = [np.array([0.5, -0.25, 2.0])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    ol.adam_step(p, g, m, v, 1, lr=0.1)
    assert np.allclose(p[0], [0.9, -1.9, 2.9], rtol=1e-7)


def test_features_partition_and_constant_frames():
    from paper_1409_4256_gb300 import synth
    det = synth.make_detector(64, 64, 0.1)
    bins = ol.feature_bins(det.q)
    assert bins.min() >= 0 and bins.max() < ol.N_FEAT
    K = np.full((2, det.q.shape[0]), 3.0)
    K[1] = 0.0
    f = ol.features(det.q, K)
    used = np.bincount(bins, minlength=ol.N_FEAT) > 0
    assert np.allclose(f[0, used], np.log(4.0)) and np.all(f[0, ~used] == 0) and np.all(f[1] == 0)
    # one photon in one pixel lands in that pixel's bin only
    K1 = np.zeros((1, det.q.shape[0]))
    K1[0, 100] = 5.0
    f1 = ol.features(det.q, K1)
    b = bins[100]
    assert np.count_nonzero(f1) == 1 and np.isclose(f1[0, b], np.log1p(5.0 / (bins == b).sum()))
    # the angular bins turn with an in-plane rotation of the detector by 2 pi / 16
    a = 2 * np.pi / 16
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    qr = det.q @ Rz.T
    bins_r = ol.feature_bins(qr)
    same_r = (bins_r // 16) == (bins // 16)
    assert same_r.mean() > 0.99


def test_topm_is_the_top_set():
    rng = np.random.default_rng(1)
    z = rng.normal(size=(5, 300))
    c = ol.topm(z, 17)
    for r in range(5):
        assert set(c[r]) == set(np.argpartition(-z[r], 17)[:17])


def test_sparse_steps_reduce_to_dense(oracle):
    rng = np.random.default_rng(2)
    n_rot, n_pix, n_data = 9, 11, 6
    W = rng.uniform(0.2, 3, size=(n_rot, n_pix))
    w = np.full(n_rot, 1 / n_rot)
    K = rng.poisson(1.0, size=(n_data, n_pix)).astype(float)
    S = oracle.scores(W, w, K)
    P, lse, _ = oracle.estep(S)
    allc = np.tile(np.arange(n_rot), (n_data, 1))
    Pc, lsec = ol.sparse_estep(S, allc)
    assert np.allclose(Pc, P.T, rtol=1e-12) and np.allclose(lsec, lse, rtol=1e-13)
    Num, den = oracle.mstep(P, K)
    Ns, ds = ol.sparse_mstep(Pc, allc, K, n_rot)
    assert np.allclose(Ns, Num, rtol=1e-12) and np.allclose(ds, den, rtol=1e-12)
    assert np.allclose(ol.missed_mass(P, allc), 0.0, atol=1e-12)
    # a strict subset: responsibilities renormalise over it and the missed
    # mass is what the dense posterior puts outside
    sub = np.sort(np.argsort(-S, axis=0)[:4].T, axis=1)
    Pc4, _ = ol.sparse_estep(S, sub)
    assert np.allclose(Pc4.sum(axis=1), 1.0)
    mm = ol.missed_mass(P, sub)
    assert np.all(mm >= -1e-15) and np.all(mm < 1)
    assert np.allclose(Pc4 * (1 - mm)[:, None], np.take_along_axis(P.T, sub, axis=1))


def test_soft_targets_renormalised():
    rng = np.random.default_rng(3)
    P = rng.random((20, 6))
    P /= P.sum(axis=0)
    idx, prob = ol.soft_targets(P, 4)
    assert idx.shape == (6, 4) and np.allclose(prob.sum(axis=1), 1.0)
    assert np.all(P.T[np.arange(6), idx[:, 0]] == P.max(axis=0))


def test_merge_candidates_hand_cases():
    from oracle import learned as ol
    first = np.array([[5, 2], [0, 1]])
    rest = np.array([[2, 7, 5, 9, 3], [4, 3, 2, 1, 0]])
    out = ol.merge_candidates(first, rest, 4)
    assert out.tolist() == [[5, 2, 7, 9], [0, 1, 4, 3]]
    # every merged set holds all of `first` and M distinct entries
    rng = np.random.default_rng(40)
    first = np.stack([rng.permutation(50)[:6] for _ in range(20)])
    rest = np.stack([rng.permutation(50)[:16] for _ in range(20)])
    out = ol.merge_candidates(first, rest, 16)
    for k in range(20):
        assert set(first[k]) <= set(out[k]) and len(set(out[k])) == 16
        assert set(out[k]) <= set(first[k]) | set(rest[k])


def test_bf16_round():
    # values with at most 8 significant bits are BF16 numbers and stay put;
    # halfway cases go to the even neighbour; the error is at most half a unit
    # in the 8th significant bit, 2^-8 relative;
    # and it agrees with PyTorch's own float -> bfloat16 conversion on the CPU
    from oracle.learned import bf16_round
    exact = np.array([0.0, 1.0, -3.5, 255.0, 2.0 ** -20 * 129, 1.0 + 2.0 ** -7])
    assert np.array_equal(bf16_round(exact), exact)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8)])
    assert np.array_equal(bf16_round(ties), [1.0, 1.0 + 2.0 ** -6, -1.0])
    rng = np.random.default_rng(11)
    x = rng.normal(size=20000) * np.exp(rng.uniform(-30, 30, size=20000))
    r = bf16_round(x)
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(r - x32) <= 2.0 ** -8 * np.abs(x32))
    torch = pytest.importorskip("torch")
    t = torch.as_tensor(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(r, t)


def test_rounded_mlp_reduces_to_the_fp64_one():
    # with the identity for the operand rounding the MLP is the pinned FP64 one;
    # with BF16 operands its gradients stay within the rounding's effect
    from oracle import learned as ol
    rng = np.random.default_rng(12)
    ps = []
    for fo in (16, 16, 16, 10):
        ps += [rng.normal(0, 0.3, size=(16 if ps else 16, fo)), rng.normal(0, 0.1, size=fo)]
    X = rng.uniform(0, 2, size=(6, 16))
    T = ol.dense_targets(rng.integers(0, 10, size=(6, 2)), np.full((6, 2), 0.5), 10)
    l0, g0 = ol.mlp_loss_grads(ps, X, T)
    l1, g1 = ol.mlp_loss_grads(ps, X, T, operand=lambda a: a)
    assert l0 == l1 and all(np.array_equal(a, b) for a, b in zip(g0, g1))
    l2, g2 = ol.mlp_loss_grads(ps, X, T, operand=ol.bf16_round)
    assert abs(l2 - l0) <= 1e-2 * abs(l0)
    for a, b in zip(g2, g0):
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b)
