"""Sparse-K form of the E-step pass 1 against the FP64 oracle.

The scores are Eq. 2.3's sum_i K_ik log W_ij + bias_j taken over each frame's
non-zero pixels only, which is the definition itself (zero counts contribute
nothing), so the oracle is the dense one. Bars as for the FP32 form: lse within
1e-4, and the dense FP32 pass 1 of the same context agrees to 1e-5.
Problem: the small ragged problem with one empty frame and one frame holding
a single large count.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4256_gb300 import build
    build.build()
    return torch


def test_sparse_k_matches_oracle_and_dense(torch_cuda, oracle, small_problem):
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    K = p["K"].copy()
    K[7] = 0
    K[11] = 0
    K[11, 300] = 200
    nrot, nd = p["quat"].shape[0], K.shape[0]
    W = oracle.expand(p["grid"], p["quat"], p["q"], p["w_floor"])
    _, lse_o, _ = oracle.estep(oracle.scores(W, p["w"], K.astype(np.float64)))
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision="fp32",
                      w_floor=p["w_floor"], sparse_k=True)
    ctx.set_frames(torch.as_tensor(K, device="cuda"))
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(g, 0, nrot)
    m, s = ctx.loglik_sparse_k(L, bias, nrot)
    md, sd = ctx.loglik(L, bias, nrot)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    lse = (m + torch.log(s)).cpu().numpy()[:nd]
    lse_d = (md + torch.log(sd)).cpu().numpy()[:nd]
    assert np.abs(lse - lse_o).max() <= 1e-4
    assert np.abs(lse - lse_d).max() <= 1e-5


def test_sparse_k_accumulates_over_rotation_blocks(torch_cuda, small_problem):
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision="fp32",
                      w_floor=p["w_floor"], sparse_k=True)
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(g, 0, nrot)
    m_all, s_all = ctx.loglik_sparse_k(L, bias, nrot)
    m = torch.empty_like(m_all)
    s = torch.empty_like(s_all)
    for r0 in range(0, nrot, 512):  # 1380 rotations: blocks of 512, 512, 356
        nb = min(512, nrot - r0)
        Lb, bb = ctx.expand(g, r0, nb)
        ctx.loglik_sparse_k(Lb, bb, nb, m, s, accumulate=r0 > 0)
    torch.cuda.synchronize()
    a = (m_all + torch.log(s_all)).cpu().numpy()[:nd]
    b = (m + torch.log(s)).cpu().numpy()[:nd]
    assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max() + 1e-9
