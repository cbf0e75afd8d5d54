"""The boundary's failure statuses (the device status word read by
emc_ctx_status) on the GPU, caused without faulting or hanging it:

* EMC_ERR_TIMEOUT: the context's stall hook (emc_ctx_set_wait_limit) makes the
  MMA issuer of every tensor-core launch wait on a barrier that nothing
  completes, with a 1 ms limit. The wait runs out, the kernel records the
  status, lets the copies it issued land, frees its tensor memory and returns.
  The same context then computes the oracle's results with the hook cleared.
* EMC_ERR_NUMERIC: a NaN or an infinity planted in the model on the host
  reaches the expansion (Eq. 2.9), which flags the non-finite W_ij.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TIMEOUT, NUMERIC = -5, -6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4256_gb300 import build
    build.build()
    return torch


def _ctx(torch, p, precision="bf16_split", **kw):
    from paper_1409_4256_gb300 import emc
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], p["K"].shape[0], precision=precision,
                      w_floor=p["w_floor"], **kw)
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    return ctx


@pytest.fixture(scope="module")
def ref(small_problem, oracle):
    p = small_problem
    W = oracle.expand(p["grid"], p["quat"], p["q"], p["w_floor"])
    P, lse, _ = oracle.estep(oracle.scores(W, p["w"], p["K"].astype(np.float64)))
    out, _, L = oracle.iteration(p["grid"], p["quat"], p["w"], p["q"], p["K"].astype(np.float64),
                                 p["w_floor"])
    return dict(lse=lse, out=out, L=L)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_timeout_in_pass1_then_recovery(torch_cuda, small_problem, ref):
    torch, p = torch_cuda, small_problem
    ctx = _ctx(torch, p)
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(g, 0, nrot)
    ctx.set_wait_limit(1_000_000, stall=True)  # 1 ms
    ctx.loglik(L, bias, nrot)
    torch.cuda.synchronize()  # the launch returned
    assert ctx.status() == TIMEOUT
    ctx.set_wait_limit(0, stall=False)
    m, s = ctx.loglik(L, bias, nrot)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    lse = (m + torch.log(s)).cpu().numpy()[:nd]
    assert np.abs(lse - ref["lse"]).max() <= 1e-4


def test_timeout_in_bound_pass_then_recovery(torch_cuda, small_problem, ref):
    # every tensor-core launch of a bound-pruned iteration stalls (the bound,
    # the exact pass 1, the normalisation); the iteration still returns
    torch, p = torch_cuda, small_problem
    ctx = _ctx(torch, p, store_scores=False)
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    _, st = ctx.iteration(g)  # dense: gives the frame order
    assert st["device_status"] == 0
    ctx.set_wait_limit(1_000_000, stall=True)
    _, st = ctx.iteration(g)
    assert st["pass1_pruned"] == 1 and st["device_status"] == TIMEOUT
    assert ctx.status() == TIMEOUT
    ctx.set_wait_limit(0, stall=False)
    out, st = ctx.iteration(g)
    assert st["device_status"] == 0 and ctx.status() == 0
    assert _rel(out.cpu().numpy().astype(np.float64), ref["out"]) <= 1e-5
    assert abs(st["loglik"] - ref["L"]) <= 1e-4 * p["K"].shape[0]


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("precision", ["fp32", "bf16_split"])
def test_non_finite_model_is_flagged(torch_cuda, small_problem, ref, bad, precision):
    torch, p = torch_cuda, small_problem
    ctx = _ctx(torch, p, precision)
    N, nrot = p["N"], p["quat"].shape[0]
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    gb = g.clone()
    c = N // 2
    gb[c - 1:c + 2, c - 1:c + 2, c - 1:c + 2] = bad  # every slice passes the centre
    ctx.expand(gb, 0, nrot)
    torch.cuda.synchronize()
    assert ctx.status() == NUMERIC
    _, st = ctx.iteration(gb)
    assert st["device_status"] == NUMERIC
    assert ctx.status() == NUMERIC
    out, st = ctx.iteration(g)  # a finite model again: the context is usable
    assert st["device_status"] == 0
    assert _rel(out.cpu().numpy().astype(np.float64), ref["out"]) <= 1e-5
