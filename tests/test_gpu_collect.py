"""Responsibilities recorded during emc_iteration (emc_set_collect) and the
targets and missed mass drawn from them (emc_collected_targets), against the
FP64 oracle's P of the same iteration (Eq. 2.4) and against the calls that read
stored scores.

Recording reads the blocks of P the M-step contracts, so it works where the
scores are recomputed in pass 2 and where pass 1 is bound-pruned. The targets
are the R rotations of largest P_jk with weights P_jk over their sum (the
softmax of their scores); the missed mass is the P_jk outside the frame's
candidate set."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

R = 8
M = 64
UNSUPPORTED = -4  # EMC_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_4256_gb300 import build
    build.build()
    return torch


def _oracle_P(oracle, p, g, model):
    K = p["K"].astype(np.float64)
    if model == "poisson":
        _, _, _, P = oracle.iteration(g, p["quat"], p["w"], p["q"], K, p["w_floor"], want_P=True)
    else:
        _, _, _, P = oracle.iteration_poisson_fluence(g, p["quat"], p["w"], p["q"], K,
                                                      p["w_floor"], want_P=True)
    return P  # [n_rot, n_data]


def _candidates(P, seed):
    # per frame: the oracle's 4 best rotations and random others, distinct
    rng = np.random.default_rng(seed)
    nrot, nd = P.shape
    out = np.empty((nd, M), dtype=np.int32)
    for k in range(nd):
        top = list(np.argsort(-P[:, k], kind="stable")[:4])
        rest = [j for j in rng.permutation(nrot) if j not in top][:M - 4]
        out[k] = np.array(top + rest, dtype=np.int32)
    return out


def _check_targets(tidx, tprob, P, thr=1e-5, tol=2e-4):
    nrot, nd = P.shape
    for k in range(nd):
        assert len(set(tidx[k].tolist())) == R  # distinct, fill included
        assert np.all((tidx[k] >= 0) & (tidx[k] < nrot))
        order = sorted(range(nrot), key=lambda j: (-P[j, k], j))[:R]
        w = P[order, k] / P[order, k].sum()
        want = {j: x for j, x in zip(order, w) if x > thr}
        got = {int(j): float(x) for j, x in zip(tidx[k], tprob[k]) if x > thr}
        assert want.keys() == got.keys(), (k, want, got)
        assert all(abs(want[j] - got[j]) <= tol for j in want)
        assert abs(float(tprob[k].sum()) - 1.0) <= 1e-5


@pytest.mark.parametrize("model,precision,stored,dense", [
    ("poisson", "bf16_split", True, False), ("poisson", "bf16_split", False, False),
    ("poisson", "bf16_split", True, True), ("poisson", "fp16_split", True, False),
    ("poisson", "bf16", True, True), ("poisson_fluence", "bf16_split", False, False)])
def test_collected_targets_and_missed_mass(torch_cuda, oracle, small_problem, model, precision,
                                           stored, dense):
    from paper_1409_4256_gb300 import emc
    torch, p = torch_cuda, small_problem
    nd = p["K"].shape[0]
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision=precision,
                      w_floor=p["w_floor"], store_scores=stored, dense_estep=dense, model=model,
                      n_cand=M)
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    # room for every rotation of every frame: near the start model many
    # rotations per frame keep a non-zero P on this small problem
    ctx.collect(p["quat"].shape[0])
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    g1, _ = ctx.iteration(g)  # the first call on fresh frames runs the dense pass
    gin = g1.double().cpu().numpy()
    P = _oracle_P(oracle, p, gin, model)
    cand = _candidates(P, 5)
    ctx.set_candidates(torch.as_tensor(cand, device="cuda"))
    _, st = ctx.iteration(g1)  # pruned where the context prunes
    assert st["device_status"] == 0
    if not dense and precision != "bf16":
        assert st["pass1_pruned"] == 1
    tidx, tprob, mm = (x.cpu().numpy() for x in ctx.collected_targets(R, missed=True))
    assert ctx.status() == 0
    # the split forms against the oracle at the 1e-4 bar on P; plain BF16's P
    # is itself off by up to one BF16 rounding of log W per element (2^-8 of
    # |S_jk - lse_k|), so it is held to its own stored-score calls below, where
    # the recorded P (BF16, 2^-8 relative) is the only difference
    tol, thr = (1e-2, 1e-3) if precision == "bf16" else (2e-4, 1e-5)
    if precision != "bf16":
        _check_targets(tidx, tprob, P, thr=thr, tol=tol)
        want_mm = np.array([P[np.setdiff1d(np.arange(P.shape[0]), cand[k]), k].sum()
                            for k in range(nd)])
        assert np.abs(mm - want_mm).max() <= tol
    if stored:  # the stored-score calls on the same iteration
        ts, ps = (x.cpu().numpy() for x in ctx.targets_from_scores(R))
        for k in range(nd):
            a = {int(j): float(x) for j, x in zip(tidx[k], tprob[k]) if x > thr}
            b = {int(j): float(x) for j, x in zip(ts[k], ps[k]) if x > thr}
            assert a.keys() == b.keys() and all(abs(a[j] - b[j]) <= tol for j in a)
        ms = ctx.missed_mass().cpu().numpy()
        assert np.abs(mm - ms).max() <= tol


def test_collect_stops_overflows_and_rejects(torch_cuda, small_problem):
    from paper_1409_4256_gb300 import emc
    torch, p = torch_cuda, small_problem
    nd = p["K"].shape[0]
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")

    def ctx(**kw):
        c = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, w_floor=p["w_floor"], **kw)
        c.set_frames(torch.as_tensor(p["K"], device="cuda"))
        return c

    a = ctx(precision="bf16_split", store_scores=True)
    with pytest.raises(emc.EmcError):  # nothing recorded yet
        a.collected_targets(R)
    a.collect(p["quat"].shape[0])
    with pytest.raises(emc.EmcError):  # still nothing: no iteration since
        a.collected_targets(R)
    a.iteration(g)
    tidx, _ = a.collected_targets(R)
    assert a.status() == 0
    # one entry per frame cannot hold the frames' non-zero responsibilities
    # (from the start model: many per frame)
    a.collect(1)
    a.iteration(g)
    a.collected_targets(R)
    assert a.status() == UNSUPPORTED
    a.collect(0)  # stopped: the next iteration records nothing
    a.iteration(g)
    with pytest.raises(emc.EmcError):
        a.collected_targets(R)
    # FP32 and the Gaussian model are not recorded
    for kw in (dict(precision="fp32"), dict(precision="fp16_split", model="gaussian", sigma=1.0)):
        with pytest.raises(emc.EmcError):
            ctx(**kw).collect(32)
