"""GPU parity of the learned proposal and the sparse Maximize against the
FP64 oracle (oracle/learned.py, oracle/emc_oracle.c) on the same inputs.

Tolerances: features 1e-5 absolute (FP32 log1p of exact bin sums); MLP logits,
loss and gradients rel-L2 1e-2 against the FP64 oracle (the products take
BF16-rounded operands, unit roundoff 2^-8: measured on the CPU, that rounding
alone moves them by 5e-3 to 6e-3 rel-L2 at K = 512) and 1e-3 against the
oracle with the same operand rounding (what remains is FP32 accumulation and
the FP32 GELU, plus operands that land on the other side of a BF16 rounding);
sparse responsibilities max|dP| <= 1e-4, lse 1e-4, model rel-L2 <= 1e-5 (the
same bar as the dense forms, same exact score split)."""
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


@pytest.fixture(scope="module")
def dense_ref(small_problem, oracle):
    p = small_problem
    W = oracle.expand(p["grid"], p["quat"], p["q"], p["w_floor"])
    S = oracle.scores(W, p["w"], p["K"].astype(np.float64))
    P, lse, L = oracle.estep(S)
    return dict(W=W, S=S, P=P, lse=lse)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def ctx_for(torch, p, precision="bf16_split", n_cand=0, store_scores=False, sparse_k=False):
    from paper_1409_4256_gb300 import emc
    c = emc.Context(p["N"], p["q"], p["quat"], p["w"], p["K"].shape[0], precision=precision,
                    w_floor=p["w_floor"], n_cand=n_cand, store_scores=store_scores,
                    sparse_k=sparse_k)
    c.set_frames(torch.as_tensor(p["K"], device="cuda"))
    return c


@pytest.mark.parametrize("precision", ["bf16_split", "fp16_split"])
def test_features(torch_cuda, small_problem, precision):
    from oracle import learned as ol
    torch, p = torch_cuda, small_problem
    ctx = ctx_for(torch, p, precision)
    f = ctx.features()
    torch.cuda.synchronize()
    nd = p["K"].shape[0]
    ref = ol.features(p["q"], p["K"])
    got = f.cpu().numpy()
    assert np.abs(got[:nd] - ref).max() < 1e-5
    assert np.all(got[nd:] == 0)


def _oracle_params(torch, prop):
    from oracle import learned as ol
    y = prop.params.cpu().numpy().astype(np.float64)
    H, ld = 512, prop.ld_out
    ps, o = [], 0
    for l in range(4):
        out = H if l < 3 else ld
        ps.append(y[o:o + H * out].reshape(H, out))
        o += H * out
        ps.append(y[o:o + out])
        o += out
    ps[6] = ps[6][:, :prop.n_out]
    ps[7] = ps[7][:prop.n_out]
    return ps


@pytest.mark.parametrize("B", [64, 128])
def test_mlp_forward_and_gradients(torch_cuda, B):
    # B = 64: SIMT products; B = 128: the output layer on the tensor cores
    from oracle import learned as ol
    from paper_1409_4256_gb300 import emc, learned
    torch = torch_cuda
    n_out, R = 300, 8
    prop = learned.Proposal(n_out)
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 2, size=(B, 512)).astype(np.float32)
    tidx = np.stack([rng.choice(n_out, R, replace=False) for _ in range(B)]).astype(np.int32)
    tprob = rng.random((B, R)).astype(np.float32)
    tprob /= tprob.sum(axis=1, keepdims=True)
    Xd = torch.as_tensor(X, device="cuda")
    ps = _oracle_params(torch, prop)
    # forward
    z = prop.logits(Xd, batch=B).cpu().numpy()[:, :n_out]
    zr, _ = ol.mlp_forward(ps, X.astype(np.float64))
    zb, _ = ol.mlp_forward(ps, X.astype(np.float64), operand=ol.bf16_round)
    assert rel_l2(z, zr) < 1e-2
    assert rel_l2(z, zb) < 1e-3
    # one training step: loss and the gradients it used
    work = torch.empty(emc.mlp_work_size(n_out, B), dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    emc.mlp_train_step(n_out, prop.params, prop.grads, prop.m, prop.v, 1, 1e-3, Xd,
                       torch.as_tensor(tidx, device="cuda"), torch.as_tensor(tprob, device="cuda"),
                       B, R, work, loss)
    torch.cuda.synchronize()
    T = ol.dense_targets(tidx, tprob.astype(np.float64), n_out)
    lr_, gr = ol.mlp_loss_grads(ps, X.astype(np.float64), T)
    lb_, gb_ = ol.mlp_loss_grads(ps, X.astype(np.float64), T, operand=ol.bf16_round)
    assert abs(loss.item() - lr_) < 1e-2 * abs(lr_)
    assert abs(loss.item() - lb_) < 1e-3 * abs(lb_)
    g = prop.grads.cpu().numpy().astype(np.float64)
    H, ld = 512, prop.ld_out
    o = 0
    for l in range(4):
        out = H if l < 3 else ld
        gw = g[o:o + H * out].reshape(H, out)
        o += H * out
        gb = g[o:o + out]
        o += out
        cols = out if l < 3 else n_out
        assert rel_l2(gw[:, :cols], gr[2 * l]) < 1e-2, l
        assert rel_l2(gb[:cols], gr[2 * l + 1]) < 1e-2, l
        assert rel_l2(gw[:, :cols], gb_[2 * l]) < 1e-3, l
        assert rel_l2(gb[:cols], gb_[2 * l + 1]) < 1e-3, l
        if l == 3:
            assert np.all(gw[:, n_out:] == 0) and np.all(gb[n_out:] == 0)


def test_training_reduces_loss(torch_cuda):
    from paper_1409_4256_gb300 import learned
    torch = torch_cuda
    n_out, n = 200, 1024
    rng = np.random.default_rng(6)
    # a learnable toy: the target class is a fixed random projection's argmax
    X = rng.normal(size=(n, 512)).astype(np.float32)
    lab = np.argmax(X @ rng.normal(size=(512, n_out)), axis=1).astype(np.int32)
    prop = learned.Proposal(n_out)
    hist = prop.train(torch.as_tensor(X, device="cuda"),
                      torch.as_tensor(lab[:, None], device="cuda"),
                      torch.ones((n, 1), dtype=torch.float32, device="cuda"),
                      np.arange(n), epochs=6, batch=128, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0]


def test_topm_matches_sorting(torch_cuda):
    from oracle import learned as ol
    from paper_1409_4256_gb300 import emc
    torch = torch_cuda
    rng = np.random.default_rng(7)
    B, n, ld, M = 37, 5000, 5056, 129
    z = rng.normal(size=(B, ld)).astype(np.float32)
    z[3, :100] = 7.0  # a block of equal values straddling the cut
    z[3, 100:] = rng.uniform(-1, 1, size=ld - 100).astype(np.float32)
    cand = torch.empty((B, M), dtype=torch.int32, device="cuda")
    emc.topm(torch.as_tensor(z, device="cuda"), B, n, ld, M, cand)
    got = np.sort(cand.cpu().numpy(), axis=1)
    ref = ol.topm(z[:, :n].astype(np.float64), M)
    assert np.array_equal(got, ref)


def test_merge_candidates_matches_oracle(torch_cuda):
    # integer work: bit-exact, including the order of the merged entries
    from oracle import learned as ol
    from paper_1409_4256_gb300 import emc
    torch = torch_cuda
    rng = np.random.default_rng(9)
    n, n_rot = 300, 4000
    for R, M_rest, M in ((32, 512, 512), (64, 100, 100), (5, 40, 33), (0, 64, 64)):
        first = np.stack([rng.permutation(n_rot)[:R] for _ in range(n)]).astype(np.int32)
        # rest overlaps first heavily: its head repeats part of first
        rest = np.stack([np.concatenate([f[:R // 2], np.setdiff1d(rng.permutation(n_rot), f)
                                         [:M_rest - R // 2]]) for f in first]).astype(np.int32)
        got = emc.merge_candidates(torch.as_tensor(first, device="cuda") if R else None,
                                   torch.as_tensor(rest, device="cuda"), M).cpu().numpy()
        assert np.array_equal(got, ol.merge_candidates(first, rest, M))
    with pytest.raises(emc.EmcError):  # rest shorter than M
        emc.merge_candidates(None, torch.zeros((4, 8), dtype=torch.int32, device="cuda"), 9)


def _candidates(dense_ref, M, seed=8):
    # the top M/2 dense scores plus M/2 random others, sorted per frame
    S = dense_ref["S"]
    rng = np.random.default_rng(seed)
    out = []
    for k in range(S.shape[1]):
        top = np.argsort(-S[:, k])[:M // 2]
        rest = rng.choice(np.setdiff1d(np.arange(S.shape[0]), top), M - M // 2, replace=False)
        out.append(np.sort(np.concatenate([top, rest])))
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("sparse_k", [False, True])
@pytest.mark.parametrize("precision", ["fp32", "bf16_split", "fp16_split"])
def test_sparse_steps(torch_cuda, small_problem, dense_ref, precision, sparse_k):
    # sparse_k: the frames' non-zero pixel lists replace their rows
    from oracle import learned as ol
    torch, p = torch_cuda, small_problem
    M = 96
    cand = _candidates(dense_ref, M)
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    ctx = ctx_for(torch, p, precision, n_cand=M, sparse_k=sparse_k)
    ctx.set_candidates(torch.as_tensor(cand, device="cuda"))
    L, bias = ctx.expand(torch.as_tensor(p["grid"].astype(np.float32), device="cuda"), 0, nrot)
    P, lse = ctx.sparse_estep(L, bias)
    Num, den = ctx.sparse_update(P)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    Pr, lser = ol.sparse_estep(dense_ref["S"], cand)
    tol = 1e-3 if precision == "fp16_split" else 1e-4  # FP16 rest term, see test_gpu_parity
    assert np.abs(P.cpu().numpy()[:nd] - Pr).max() <= tol
    assert np.abs(lse.cpu().numpy()[:nd] - lser).max() <= tol
    Nr, dr = ol.sparse_mstep(Pr, cand, p["K"], nrot)
    assert rel_l2(Num.cpu().numpy()[:nrot, :p["q"].shape[0]], Nr) <= 1e-4
    assert rel_l2(den.cpu().numpy()[:nrot], dr) <= 1e-4


@pytest.mark.parametrize("sparse_k", [False, True])
def test_sparse_iteration_matches_oracle(torch_cuda, small_problem, dense_ref, oracle, sparse_k):
    from oracle import learned as ol
    torch, p = torch_cuda, small_problem
    M = 96
    cand = _candidates(dense_ref, M, seed=9)
    nrot = p["quat"].shape[0]
    Pr, _ = ol.sparse_estep(dense_ref["S"], cand)
    Nr, dr = ol.sparse_mstep(Pr, cand, p["K"], nrot)
    want, _, _ = oracle.compress(p["N"], p["quat"], p["q"], Nr, dr, p["grid"])
    ctx = ctx_for(torch, p, "bf16_split", n_cand=M, sparse_k=sparse_k)
    ctx.set_candidates(torch.as_tensor(cand, device="cuda"))
    out, st = ctx.sparse_iteration(torch.as_tensor(p["grid"].astype(np.float32), device="cuda"))
    assert st["device_status"] == 0
    assert rel_l2(out.cpu().numpy().astype(np.float64), want) <= 1e-5


def test_all_rotations_as_candidates_is_the_dense_iteration(torch_cuda, small_problem):
    torch, p = torch_cuda, small_problem
    nrot, nd = p["quat"].shape[0], p["K"].shape[0]
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    dense, _ = ctx_for(torch, p, "bf16_split").iteration(g)
    ctx = ctx_for(torch, p, "bf16_split", n_cand=nrot)
    ctx.set_candidates(torch.arange(nrot, dtype=torch.int32, device="cuda").repeat(nd, 1))
    sparse, st = ctx.sparse_iteration(g)
    assert rel_l2(sparse.cpu().numpy().astype(np.float64),
                  dense.cpu().numpy().astype(np.float64)) < 1e-6


def test_targets_and_missed_mass(torch_cuda, small_problem, dense_ref):
    from oracle import learned as ol
    torch, p = torch_cuda, small_problem
    M, R = 64, 16
    cand = _candidates(dense_ref, M, seed=10)
    nd = p["K"].shape[0]
    ctx = ctx_for(torch, p, "bf16_split", n_cand=M, store_scores=True)
    ctx.set_candidates(torch.as_tensor(cand, device="cuda"))
    ctx.iteration(torch.as_tensor(p["grid"].astype(np.float32), device="cuda"))
    tidx, tprob = ctx.targets_from_scores(R)
    missed = ctx.missed_mass()
    torch.cuda.synchronize()
    ridx, rprob = ol.soft_targets(dense_ref["P"], R)
    gi, gp = tidx.cpu().numpy(), tprob.cpu().numpy()
    for k in range(nd):
        o = np.argsort(gi[k])
        q = np.argsort(ridx[k])
        assert np.array_equal(gi[k][o], ridx[k][q])
        assert np.abs(gp[k][o] - rprob[k][q]).max() < 1e-4
    mr = ol.missed_mass(dense_ref["P"], cand)
    assert np.abs(missed.cpu().numpy() - mr).max() < 1e-4


def test_trained_proposal_beats_untrained(torch_cuda, oracle):
    """What the network gains: the responsibility mass its top-M candidates
    capture on held-out frames, trained vs. the same network untrained."""
    from paper_1409_4256_gb300 import emc, learned, synth
    torch = torch_cuda
    ds = synth.make_dataset(32, 32, 3000, 2.0, radius=8.0)
    quat, w = emc.quat_generate(3)
    grid = torch.as_tensor(ds.model_true.astype(np.float32), device="cuda")
    M = 64
    ctx = emc.Context(32, ds.q, quat, w, ds.K.shape[0], precision="bf16_split",
                      w_floor=1e-10 * float(ds.model_true.mean()), n_cand=M, store_scores=True)
    ctx.set_frames(torch.as_tensor(ds.K, device="cuda"))
    ctx.iteration(grid)
    tidx, tprob = ctx.targets_from_scores(16)
    feat = ctx.features()
    train, test = learned.split_rows(ds.K.shape[0])
    nrot = quat.shape[0]

    def recall(prop):
        cand = prop.propose(feat, M, ds.K.shape[0])
        ctx.set_candidates(cand)
        mm = ctx.missed_mass().cpu().numpy()
        return float(1.0 - mm[test].mean())

    prop = learned.Proposal(nrot)
    before = recall(prop)
    hist = prop.train(feat, tidx, tprob, train, epochs=30, batch=256, lr=1e-3)
    after = recall(prop)
    assert hist[-1] < hist[0]
    assert after > before + 0.1 and after > 2 * M / nrot, (before, after, hist[0], hist[-1])


def test_schedules_with_and_without_the_network(torch_cuda):
    """The learned schedule against the same schedule without the network, at
    equal M: candidates = the last dense E-step's top R plus the network's best
    others, plus random rotations instead, or the dense E-step's own top M;
    4 sparse iterations per dense one, 10 iterations from the same model. Each
    is held to the target's 1e-3 (model rel-L2 against the dense iterations);
    the printed missed mass at the dense steps shows what each set leaves out."""
    from paper_1409_4256_gb300 import emc, learned, synth
    torch = torch_cuda
    ds = synth.make_dataset(32, 32, 3000, 2.0, radius=8.0)
    quat, w = emc.quat_generate(3)
    nrot, nd, M, R = quat.shape[0], ds.K.shape[0], 64, 8
    floor = 1e-10 * float(ds.model_start.mean())
    Kd = torch.as_tensor(ds.K, device="cuda")
    ctx = emc.Context(32, ds.q, quat, w, nd, precision="bf16_split", w_floor=floor, n_cand=M,
                      store_scores=True)
    dense = emc.Context(32, ds.q, quat, w, nd, precision="bf16_split", w_floor=floor)
    for c in (ctx, dense):
        c.set_frames(Kd)
    g0 = torch.as_tensor(ds.model_start.astype(np.float32), device="cuda")
    g1, _ = ctx.iteration(g0)
    g2, _ = ctx.iteration(g1)
    tidx, tprob = ctx.targets_from_scores(16)
    feat = ctx.features()
    train, test = learned.split_rows(nd)
    prop = learned.Proposal(nrot)
    prop.train(feat, tidx, tprob, train, epochs=30, batch=256, lr=1e-3)
    net = prop.propose(feat, M, nd)
    rng = np.random.default_rng(1008)
    offs = np.sort(rng.choice(nrot, M, replace=False))
    rand = torch.as_tensor(((rng.integers(0, nrot, size=nd)[:, None] + offs[None, :]) % nrot)
                           .astype(np.int32), device="cuda")
    frames = torch.arange(nd, dtype=torch.int32, device="cuda")

    def dense_top_m():
        cand = torch.empty((nd, M), dtype=torch.int32, device="cuda")
        emc.topm(ctx.responsibilities(frames), nd, nrot, nrot, M, cand)
        return cand

    refresh = {
        "network": lambda: emc.merge_candidates(ctx.targets_from_scores(R)[0], net, M),
        "random_filler": lambda: emc.merge_candidates(ctx.targets_from_scores(R)[0], rand, M),
        "dense_top_m": dense_top_m}
    a, b = g2.clone(), torch.empty_like(g2)
    for _ in range(10):
        dense.iteration(a, b)
        a, b = b, a
    ref = a.double()
    out = {}
    for name, make in refresh.items():
        ctx.iteration(g2)
        ctx.set_candidates(make())
        c, d = g2.clone(), torch.empty_like(g2)
        missed = []
        for it in range(10):
            if it % 5 == 4:
                ctx.iteration(c, d)
                missed.append(float(ctx.missed_mass().mean().item()))
                ctx.set_candidates(make())
            else:
                ctx.sparse_iteration(c, d)
            c, d = d, c
        diff = float(torch.linalg.norm(c.double() - ref) / torch.linalg.norm(ref))
        out[name] = (diff, missed)
    print("\nschedules at 32^3 (1380 rotations, 3000 frames, M = 64, dense top 8 kept): " +
          ", ".join(f"{k}: model rel-L2 vs dense {v[0]:.2e}, missed mass {v[1]}"
                    for k, v in out.items()))
    for name in out:
        assert out[name][0] <= 1e-3, (name, out[name])
