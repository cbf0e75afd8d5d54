"""Parity at the workloads' full sizes, on outputs the oracle can compute one
by one and on identities that hold at any size.

* emc64 (64^3, 64x64 detector with 10% masked, n=10 -> 50100 rotations, 20000
  frames), the benchmark's configuration: every step over all rotations at
  once (the tile and launch shapes emc_iteration uses, scores stored).
* emc128 (128^3, 128x128 detector, n=16 -> 204960 rotations, 100000 frames):
  the same steps over rotation blocks of 8192 (merging lse across blocks).

Sampled outputs: lse_k and the column P_{.k} of a few frames, against the FP64
oracle's scores of those frames over every rotation. Identities (exact in
real arithmetic, checked to FP32-accumulation accuracy):
  sum_j P_jk = 1 per frame            -> sum_j den_j = M_data
  sum_{i<n_pix} Num_ij = sum_k P_jk N_k  -> sum_ij Num_ij = sum_k N_k (photons)
  trilinear weights of an interior point sum to 1
                                      -> sum_l g_den_l = n_pix sum_j den_j,
                                         sum_l g_num_l = sum_ij Num_ij.
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


def _oracle_columns(oracle, grid, quat, w, q, Ks, floor, chunk=4096):
    """FP64 scores of the sampled frames Ks against every rotation -> (lse, P)."""
    S = np.empty((quat.shape[0], Ks.shape[0]))
    for j0 in range(0, quat.shape[0], chunk):
        W = oracle.expand(grid, quat[j0:j0 + chunk], q, floor)
        S[j0:j0 + chunk] = oracle.scores(W, w[j0:j0 + chunk], Ks)
    P, lse, _ = oracle.estep(S)
    return lse, P


def _run(torch, oracle, name, block, sample):
    from paper_1409_4256_gb300 import emc, synth
    cfg = synth.WORKLOADS[name]
    ds = synth.make_dataset(cfg["N"], cfg["D"], cfg["n_data"], cfg["mean_photons"],
                            masked_fraction=cfg["masked_fraction"], device="cuda")
    quat, w = emc.quat_generate(cfg["n_quat"])
    nrot, nd, npix = quat.shape[0], ds.K.shape[0], ds.q.shape[0]
    grid32 = ds.model_start.astype(np.float32)
    floor = 1e-10 * float(ds.model_start.mean())
    ctx = emc.Context(cfg["N"], ds.q, quat, w, nd, precision="bf16_split", w_floor=floor,
                      rot_chunk=block)
    ctx.set_frames(torch.as_tensor(ds.K, device="cuda"))
    g = torch.as_tensor(grid32, device="cuda")
    lse_m = torch.empty(ctx.ld_data, dtype=torch.float64, device="cuda")
    lse_s = torch.empty_like(lse_m)
    # E-step pass 1 over rotation blocks, stored scores per block
    for r0 in range(0, nrot, block):
        nb = min(block, nrot - r0)
        L, bias = ctx.expand(g, r0, nb)
        ctx.loglik(L, bias, nb, lse_m, lse_s, accumulate=r0 > 0)
        del L, bias
    # pass 2, update, compress per block; sampled P columns kept
    Pcols = np.empty((nrot, len(sample)))
    den_sum = 0.0
    num_sum = 0.0
    g_num = torch.zeros((cfg["N"],) * 3, dtype=torch.float64, device="cuda")
    g_den = torch.zeros_like(g_num)
    sidx = torch.as_tensor(sample, device="cuda")
    for r0 in range(0, nrot, block):
        nb = min(block, nrot - r0)
        L, bias = ctx.expand(g, r0, nb)
        Sb = ctx.scores_buffer(nb)
        m2 = torch.empty_like(lse_m)
        s2 = torch.empty_like(lse_s)
        ctx.loglik(L, bias, nb, m2, s2, scores=Sb)  # the block's stored scores
        P = ctx.normalize(None, None, nb, lse_m, lse_s, scores=Sb)
        b = ctx.buffer_sizes(nb)
        planes = P.view(torch.bfloat16).view(2, b.rows, b.ld_data)
        Pcols[r0:r0 + nb] = (planes[0].index_select(1, sidx).double() +
                             planes[1].index_select(1, sidx).double())[:nb].cpu().numpy()
        Num, den = ctx.update(P, nb)
        den_sum += float(den[:nb].double().sum())
        num_sum += float(Num[:nb, :npix].double().sum())
        ctx.compress(r0, nb, Num, den, g_num, g_den, accumulate=True)
        del L, bias, Sb, P, Num, den
    torch.cuda.synchronize()
    assert ctx.status() == 0
    lse = (lse_m + torch.log(lse_s)).cpu().numpy()
    lse_o, P_o = _oracle_columns(oracle, grid32.astype(np.float64), quat, w, ds.q,
                                 ds.K[sample].astype(np.float64), floor)
    return dict(lse=lse[:nd], lse_o=lse_o, P=Pcols, P_o=P_o, den_sum=den_sum, num_sum=num_sum,
                photons=float(ds.K.astype(np.float64).sum()), nd=nd, npix=npix,
                g_num=float(g_num.sum()), g_den=float(g_den.sum()))


def _check(r, sample):
    assert np.abs(r["lse"][sample] - r["lse_o"]).max() <= 1e-4
    assert np.abs(r["P"] - r["P_o"]).max() <= 1e-4
    assert abs(r["den_sum"] - r["nd"]) <= 1e-4 * r["nd"]
    assert abs(r["num_sum"] - r["photons"]) <= 1e-4 * r["photons"]
    assert abs(r["g_den"] - r["npix"] * r["den_sum"]) <= 1e-6 * r["g_den"]
    assert abs(r["g_num"] - r["num_sum"]) <= 1e-6 * r["g_num"]


def test_fullsize_emc64(torch_cuda, oracle):
    sample = np.array([0, 7, 4321, 12345, 19999])
    r = _run(torch_cuda, oracle, "emc64", 50100, sample)
    _check(r, sample)


def test_fullsize_emc128(torch_cuda, oracle):
    sample = np.array([3, 54321, 99999])
    r = _run(torch_cuda, oracle, "emc128", 8192, sample)
    _check(r, sample)
