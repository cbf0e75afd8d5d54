"""emc_loglik_static -- the E-step pass 1 for callers that cannot allocate
device memory (a host framework that owns every allocation, a process whose
pool is already committed) -- against emc_loglik on a context with a workspace.

It runs in a file of its own that pytest collects last, so that a run which
stops at the first failure has run every other test before it. It must pass
alone in a fresh process and after the other tests (the static scratch array
keeps the previous call's contents; every call overwrites what it reads).
"""
import ctypes

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


def frames_bf16(torch, K, ld_data, ld_pix, fp16=False):
    """The documented frame layout: counts, a column of ones at n_pix, zeros
    (BF16, or FP16 for the FP16 split)."""
    n_data, n_pix = K.shape
    F = torch.zeros((ld_data, ld_pix), dtype=torch.float32, device="cuda")
    F[:n_data, :n_pix] = torch.as_tensor(K, dtype=torch.float32, device="cuda")
    F[:n_data, n_pix] = 1.0
    return F.to(torch.float16 if fp16 else torch.bfloat16).contiguous()


@pytest.mark.parametrize("precision", ["fp32", "bf16_split", "fp16_split"])
def test_loglik_static_matches_workspace_call(torch_cuda, small_problem, precision):
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision=precision,
                      w_floor=p["w_floor"])
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    grid = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(grid, 0, nrot)
    m_ref, s_ref = ctx.loglik(L, bias, nrot)
    torch.cuda.synchronize()
    lse_ref = (m_ref + torch.log(s_ref)).cpu().numpy()[:nd]
    frames = frames_bf16(torch, p["K"], ctx.ld_data, ctx.ld_pix, fp16=precision == "fp16_split")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for call in range(2):  # two calls in a row share the static scratch
        m = torch.full((ctx.ld_data,), float("nan"), dtype=torch.float64, device="cuda")
        s = torch.full((ctx.ld_data,), float("nan"), dtype=torch.float64, device="cuda")
        emc.loglik_static(ctx.cfg, L, bias, frames, nrot, m, s, device_status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        lse = (m + torch.log(s)).cpu().numpy()[:nd]
        # same kernels and inputs as the workspace call: the parity tolerance
        assert np.abs(lse - lse_ref).max() <= 1e-4, (call, np.abs(lse - lse_ref).max())


def test_loglik_static_accumulates(torch_cuda, small_problem):
    # two rotation blocks merged with accumulate=1 equal the one-block result
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision="bf16_split",
                      w_floor=p["w_floor"])
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    grid = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(grid, 0, nrot)
    m_ref, s_ref = ctx.loglik(L, bias, nrot)
    La, ba = ctx.expand(grid, 0, 700)
    Lb, bb = ctx.expand(grid, 700, nrot - 700)
    frames = frames_bf16(torch, p["K"], ctx.ld_data, ctx.ld_pix)
    m = torch.empty(ctx.ld_data, dtype=torch.float64, device="cuda")
    s = torch.empty_like(m)
    emc.loglik_static(ctx.cfg, La, ba, frames, 700, m, s)
    emc.loglik_static(ctx.cfg, Lb, bb, frames, nrot - 700, m, s, accumulate=True)
    torch.cuda.synchronize()
    d = ((m + torch.log(s)) - (m_ref + torch.log(s_ref))).cpu().numpy()[:nd]
    assert np.abs(d).max() <= 1e-4


def test_loglik_static_rejects_frames_beyond_static_scratch(torch_cuda, small_problem):
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    cfg = emc.Config(N=32, precision=emc.PREC_BF16_SPLIT, n_pix=812, n_rot=1380,
                     n_data=3_000_000, w_floor=1e-10)
    dummy = torch.zeros(256, dtype=torch.float64, device="cuda")
    rc = emc.lib().emc_loglik_static(ctypes.byref(cfg), dummy.data_ptr(), dummy.data_ptr(),
                                     dummy.data_ptr(), 1380, dummy.data_ptr(), dummy.data_ptr(),
                                     0, None, int(torch.cuda.current_stream().cuda_stream))
    assert rc == -4  # EMC_ERR_UNSUPPORTED, nothing launched


@pytest.mark.parametrize("precision", ["fp32", "bf16_split"])
def test_loglik_static_over_rotation_blocks(torch_cuda, small_problem, precision):
    # 400200 frames (the small problem's 300 repeated): the 32 MiB array holds
    # the per-tile pairs of only 384 rotations at a time, so one call runs four
    # rotation blocks -- the row offsets into L and bias past the first block,
    # the plane stride of the whole L, and the merge into the earlier blocks
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    K = np.tile(p["K"], (1334, 1))
    nrot, nd = p["quat"].shape[0], K.shape[0]
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision=precision,
                      w_floor=p["w_floor"])
    ctx.set_frames(torch.as_tensor(K, device="cuda"))
    block = (32 * 2 ** 20 // (ctx.ld_data * 12)) * 64 // 128 * 128
    rows = -(-nrot // 128) * 128
    assert 128 <= block and rows > 2 * block  # at least three blocks
    grid = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    L, bias = ctx.expand(grid, 0, nrot)
    m_ref, s_ref = ctx.loglik(L, bias, nrot)
    frames = frames_bf16(torch, K, ctx.ld_data, ctx.ld_pix)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    m = torch.full((ctx.ld_data,), float("nan"), dtype=torch.float64, device="cuda")
    s = torch.full((ctx.ld_data,), float("nan"), dtype=torch.float64, device="cuda")
    emc.loglik_static(ctx.cfg, L, bias, frames, nrot, m, s, device_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and ctx.status() == 0
    d = ((m + torch.log(s)) - (m_ref + torch.log(s_ref))).cpu().numpy()[:nd]
    assert np.abs(d).max() <= 1e-4, np.abs(d).max()
