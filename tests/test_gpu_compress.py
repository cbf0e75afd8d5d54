"""GPU parity of the c-step alone (Eq. 2.12, and Eq. 2.5 + 2.10 in IDW mode).

The compression gets the same FP64 numerators and denominators as the
oracle's (rounded once to FP32, which is what the step receives), so the only
differences are its own arithmetic: FP32 trilinear weights and products, FP32
sums of the few terms that fall on one voxel within one pixel group, FP64
reductions. Each term carries a relative error of a few 2^-24, so the grids
agree to rel-L2 <= 1e-6.

Geometries (32^3 grid, 300 rotations):
  detector  the detector sheet: every pixel group's corners fit the
            shared-memory box, so every term is merged before the reduction;
  scattered pixels drawn uniformly in a ball: a group of them spans the
            grid in z, its box exceeds the capacity and the terms are reduced
            one by one;
  edge      the detector stretched to |q| = N/2 - 0.4: corners fall outside
            the grid, so the bounds-checked form runs.
Rotations with den_j = 0 (and Num_j = 0) are mixed in: they add nothing.
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def geometry(p, kind):
    N, q = p["N"], p["q"]
    if kind == "scattered":
        rng = np.random.default_rng(71)
        x = rng.standard_normal(q.shape)
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        return x * (N / 2 - 2.0) * rng.uniform(0, 1, (q.shape[0], 1)) ** (1 / 3)
    if kind == "edge":
        return q * ((N / 2 - 0.4) / np.linalg.norm(q, axis=1).max())
    return q


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("kind", ["detector", "scattered", "edge"])
def test_compress_alone(torch_cuda, small_problem, oracle, kind, mode):
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    N = p["N"]
    q = geometry(p, kind)
    quat = p["quat"][:300]
    w = p["w"][:300] / p["w"][:300].sum()
    nrot, npix = quat.shape[0], q.shape[0]
    rng = np.random.default_rng(72)
    # photon-like numerators: heavy-tailed, many exact zeros
    Num = (rng.gamma(0.5, 4.0, (nrot, npix)) * (rng.uniform(size=(nrot, npix)) < 0.7))
    den = rng.uniform(0.2, 3.0, nrot)
    dead = rng.uniform(size=nrot) < 0.2
    den[dead] = 0.0
    Num[dead] = 0.0
    Num = Num.astype(np.float32).astype(np.float64)
    den = den.astype(np.float32).astype(np.float64)
    out, gn, gd = oracle.compress(N, quat, q, Num, den, p["grid"], mode=mode)

    ctx = emc.Context(N, q, quat, w, p["K"].shape[0], precision="fp32", w_floor=p["w_floor"],
                      compress_mode=mode)
    b = ctx.buffer_sizes(nrot)
    Nt = torch.zeros((b.rows, b.ld_pix), dtype=torch.float32)
    Nt[:nrot, :npix] = torch.as_tensor(Num, dtype=torch.float32)
    dt = torch.zeros(b.rows, dtype=torch.float32)
    dt[:nrot] = torch.as_tensor(den, dtype=torch.float32)
    g_num, g_den = ctx.compress(0, nrot, Nt.cuda(), dt.cuda())
    got = ctx.finalize(g_num, g_den, torch.as_tensor(p["grid"].astype(np.float32), device="cuda"))
    torch.cuda.synchronize()
    assert ctx.status() == 0
    assert rel_l2(g_num.cpu().numpy(), gn) <= 1e-6
    assert rel_l2(g_den.cpu().numpy(), gd) <= 1e-6
    assert rel_l2(got.cpu().numpy().astype(np.float64), out) <= 1e-6
    # the voxels touched by one side only carry weights that round to zero in
    # FP32 on the other (a fraction t within 2^-24 of 1)
    gdg = g_den.cpu().numpy()
    odd = (gdg > 0) != (gd > 0)
    assert np.all(np.maximum(gdg[odd], gd[odd]) <= 1e-6 * gd.max())


def test_compress_chunks_add_up(torch_cuda, small_problem):
    # rotation blocks accumulated into one grid equal the whole range
    torch, p = torch_cuda, small_problem
    from paper_1409_4256_gb300 import emc
    N, q, quat = p["N"], p["q"], p["quat"]
    nrot, npix = quat.shape[0], q.shape[0]
    ctx = emc.Context(N, q, quat, p["w"], p["K"].shape[0], precision="fp32",
                      w_floor=p["w_floor"])
    b = ctx.buffer_sizes(nrot)
    rng = np.random.default_rng(73)
    Nt = torch.zeros((b.rows, b.ld_pix), dtype=torch.float32)
    Nt[:nrot, :npix] = torch.as_tensor(rng.gamma(0.5, 4.0, (nrot, npix)), dtype=torch.float32)
    dt = torch.zeros(b.rows, dtype=torch.float32)
    dt[:nrot] = torch.as_tensor(rng.uniform(0.2, 3.0, nrot), dtype=torch.float32)
    Nt, dt = Nt.cuda(), dt.cuda()
    a_num, a_den = ctx.compress(0, nrot, Nt, dt)
    c_num = torch.empty_like(a_num)
    c_den = torch.empty_like(a_den)
    for r0 in range(0, nrot, 384):
        nb = min(384, nrot - r0)
        ctx.compress(r0, nb, Nt[r0:], dt[r0:], c_num, c_den, accumulate=r0 > 0)
    torch.cuda.synchronize()
    assert rel_l2(c_num.cpu().numpy(), a_num.cpu().numpy()) <= 1e-13
    assert rel_l2(c_den.cpu().numpy(), a_den.cpu().numpy()) <= 1e-13
