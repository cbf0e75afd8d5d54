"""Adaptive EMC (Sec. 3.4, Eq. 3.1) on the GPU against the FP64 oracle.

Every iteration of the GPU schedule is replayed by the oracle from the same
input grid at the same sampling level: the output grid must match to the
model bar (rel-L2 <= 1e-5), the log-likelihood to the per-frame lse bar summed
over frames (1e-4 n_data), and the refinement decision must be the one the
oracle's likelihoods give, unless |dL| lies within that tolerance of the
threshold (where either decision is correct).
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


@pytest.mark.parametrize("precision", ["bf16_split", "fp32"])
def test_adaptive_schedule_stepwise(torch_cuda, oracle, small_problem, precision):
    torch = torch_cuda
    from oracle import adaptive as oad
    from paper_1409_4256_gb300 import adaptive
    p = small_problem
    K = p["K"]
    steps = []

    def keep(st, gin, gout):
        steps.append((st, gin.double().cpu().numpy(), gout.double().cpu().numpy()))

    Kd = torch.as_tensor(K, device="cuda")
    g0 = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    _, hist = adaptive.run(p["N"], p["q"], Kd, g0, 1, 3, 7, precision=precision,
                           w_floor=p["w_floor"], K_host=K, callback=keep)
    assert len(hist) == 7 and max(h.d for h in hist) >= 2
    tol_L = 1e-4 * K.shape[0]
    prev = None
    for i, (st, gin, gout) in enumerate(steps):
        quat, w = oracle.quat_generate(st.d)
        assert st.n_rot == quat.shape[0]
        out_o, _, tot = oracle.iteration(gin, quat, w, p["q"], K, p["w_floor"])
        L_o = oad.log_likelihood(tot, K)
        assert abs(st.loglik - L_o) <= tol_L
        assert np.linalg.norm(gout - out_o) <= 1e-5 * np.linalg.norm(out_o)
        refine_o = oad.should_refine(L_o, prev) and st.d < 3
        if i + 1 < len(steps):
            refined = steps[i + 1][0].d == st.d + 1
            margin = abs(abs(L_o - prev) - 0.01 * abs(L_o)) if prev is not None else np.inf
            if margin > 2 * tol_L:
                assert refined == refine_o
            prev = None if refined else L_o
