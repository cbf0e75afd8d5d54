"""emc_iteration's bound-pruned E-step pass 1 against the dense one.

With a split precision and a Poisson model, emc_iteration bounds every
(128-rotation, 256-frame) tile's scores -- by the incremental bound from the
last iteration on the same frames and by a contraction of the hi plane alone
where that is tighter -- and contracts exactly only the tiles that can hold a
score within 110 of their frames' maxima, in pass 1 and (without stored
scores) in the recomputing pass 2; it also regroups the frames by their best
rotation after every iteration. The first call on fresh frames runs the dense
pass (no order yet); later calls prune. Skipped tiles have P = 0 in FP32 and no weight
in lse at FP64 precision, so:
  * from the same input, the log-likelihood equals the dense pass's to FP64
    summation order (1e-12 relative);
  * the model equals it to FP32 summation order in the M-step, whose frames
    are in another order (rel-L2 1e-6), and the oracle's to the usual 1e-5.
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


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _ctx(torch, p, dense, stored=True, **kw):
    from paper_1409_4256_gb300 import emc
    ctx = emc.Context(p["N"], p["q"], p["quat"], p["w"], p["K"].shape[0],
                      precision="bf16_split", w_floor=p["w_floor"], store_scores=stored,
                      dense_estep=dense, **kw)
    ctx.set_frames(torch.as_tensor(p["K"], device="cuda"))
    return ctx


@pytest.mark.parametrize("model,chunk,stored", [("poisson", 0, True), ("poisson", 384, True),
                                                ("poisson_fluence", 0, True),
                                                ("poisson", 0, False), ("poisson", 384, False),
                                                ("poisson_fluence", 384, False)])
def test_pruned_iterations_equal_dense(torch_cuda, oracle, small_problem, model, chunk, stored):
    # stored: pass 2 reads the live tiles' stored scores; otherwise it recomputes
    # the scores of the live tiles only (the form for sizes whose scores do not fit)
    torch, p = torch_cuda, small_problem
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    a = _ctx(torch, p, False, stored, model=model, rot_chunk=chunk)
    d = _ctx(torch, p, True, stored, model=model, rot_chunk=chunk)
    ga, gd = g, g
    for it in range(4):  # the first call has no frame order yet and runs dense
        oa, sa = a.iteration(ga)
        od, sd = d.iteration(gd)
        assert sa["device_status"] == 0 and sd["device_status"] == 0
        # two trajectories: their models part at FP32 rounding (M-step frame order)
        assert abs(sa["loglik"] - sd["loglik"]) <= 1e-8 * abs(sd["loglik"])
        assert _rel(oa.cpu().numpy(), od.cpu().numpy()) <= 1e-6
        if it >= 1:
            assert sa["kernels"] > sd["kernels"]  # the bound, liveness and list kernels ran
        ga, gd = oa, od
    # the same input through both (one pruned step from the dense result): the
    # same scores, hence lse to FP64 summation order
    oa, sa = a.iteration(gd)
    od, sd = d.iteration(gd)
    assert abs(sa["loglik"] - sd["loglik"]) <= 1e-12 * abs(sd["loglik"])
    assert _rel(oa.cpu().numpy(), od.cpu().numpy()) <= 1e-6
    # against the oracle from the same input
    gin = gd.double().cpu().numpy()
    if model == "poisson":
        want, _, L = oracle.iteration(gin, p["quat"], p["w"], p["q"], p["K"].astype(np.float64),
                                      p["w_floor"])
    else:
        want, _, L = oracle.iteration_poisson_fluence(gin, p["quat"], p["w"], p["q"],
                                                      p["K"].astype(np.float64), p["w_floor"])
    assert _rel(oa.cpu().numpy(), want) <= 1e-5
    assert abs(sa["loglik"] - L) <= 1e-4 * p["K"].shape[0]


@pytest.mark.parametrize("precision", ["bf16_split", "fp16_split"])
def test_targets_and_missed_mass_after_pruned_iterations(torch_cuda, small_problem, precision):
    # after pruned iterations the context's stored scores are in its internal
    # frame order and hold the live tiles only; the training targets (top R and
    # their softmax) and the missed mass read them as the dense context's
    from paper_1409_4256_gb300 import emc
    torch, p = torch_cuda, small_problem
    nd, nrot, M, R = p["K"].shape[0], p["quat"].shape[0], 64, 8
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")

    def ctx(dense):
        c = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision=precision,
                        w_floor=p["w_floor"], store_scores=True, n_cand=M, dense_estep=dense)
        c.set_frames(torch.as_tensor(p["K"], device="cuda"))
        return c

    a, d = ctx(False), ctx(True)
    rng = np.random.default_rng(7)
    cand = np.stack([rng.choice(nrot, M, replace=False) for _ in range(nd)]).astype(np.int32)
    for c in (a, d):
        c.set_candidates(torch.as_tensor(cand, device="cuda"))
        for _ in range(3):  # the second and third iterations are bound-pruned in `a`
            _, st = c.iteration(g)
            assert st["device_status"] == 0
    ta, pa = (x.cpu().numpy() for x in a.targets_from_scores(R))
    td, pd = (x.cpu().numpy() for x in d.targets_from_scores(R))
    for k in range(nd):
        big_a = {int(j): float(q) for j, q in zip(ta[k], pa[k]) if q > 1e-6}
        big_d = {int(j): float(q) for j, q in zip(td[k], pd[k]) if q > 1e-6}
        assert big_a.keys() == big_d.keys()
        assert all(abs(big_a[j] - big_d[j]) <= 1e-6 for j in big_d)
    # the missed mass of the same candidate sets
    ma, md = a.missed_mass().cpu().numpy(), d.missed_mass().cpu().numpy()
    assert np.abs(ma - md).max() <= 1e-6


def _same_input_check(a, d, g):
    """One step of each context from the same input: lse to FP64 summation
    order, the model to FP32 summation order of the M-step."""
    oa, sa = a.iteration(g)
    od, sd = d.iteration(g)
    assert sa["device_status"] == 0 and sd["device_status"] == 0
    assert abs(sa["loglik"] - sd["loglik"]) <= 1e-12 * abs(sd["loglik"])
    assert _rel(oa.cpu().numpy(), od.cpu().numpy()) <= 1e-6
    return oa, sa


@pytest.mark.parametrize("precision", ["bf16_split", "fp16_split"])
def test_incremental_bound_on_reloaded_frames(torch_cuda, small_problem, precision):
    # From the second pruned iteration on the same frames the incremental bound
    # runs first (pass1_delta). Loading the same counts again changes nothing
    # (context b, reloaded, takes the same steps as a); other counts void the
    # bound for one iteration, so the hi-plane bound covers every pair of row
    # tiles. Every step equals the dense pass from the same input.
    from paper_1409_4256_gb300 import emc
    torch, p = torch_cuda, small_problem
    nd = p["K"].shape[0]

    def ctx(dense):
        c = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision=precision,
                        w_floor=p["w_floor"], store_scores=True, dense_estep=dense)
        c.set_frames(torch.as_tensor(p["K"], device="cuda"))
        return c

    a, b, d = ctx(False), ctx(False), ctx(True)
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    g1, s1 = a.iteration(g)
    b.iteration(g)
    assert s1["pass1_pruned"] == 0
    g2, s2 = _same_input_check(a, d, g1)
    _, t2 = b.iteration(g1)
    assert s2["pass1_pruned"] == 1 and s2["pass1_delta"] == 1
    b.set_frames(torch.as_tensor(p["K"], device="cuda"))  # the same counts again
    g3, s3 = _same_input_check(a, d, g2)
    _, t3 = b.iteration(g2)
    assert t3["pass1_delta"] == 1 and abs(t3["loglik"] - s3["loglik"]) <= 1e-12 * abs(s3["loglik"])
    for key in ("pass1_bound_pairs", "pass1_exact"):
        assert t3[key] == s3[key] and t2[key] == s2[key]
    # other counts: the frames of the dense context change the same way
    npairs = ((p["quat"].shape[0] + 127) // 128 + 1) // 2 * (-(-nd // 256))
    K2 = np.roll(p["K"], 1, axis=0)
    for c in (a, d):
        c.set_frames(torch.as_tensor(K2, device="cuda"))
    g4, s4 = _same_input_check(a, d, g3)
    assert s4["pass1_bound_pairs"] == npairs
    _, s5 = _same_input_check(a, d, g4)
    assert s5["pass1_delta"] == 1


def test_incremental_bound_across_sparse_iterations(torch_cuda, small_problem):
    # the learned schedule's sparse iterations expand into the other L buffer:
    # the next dense iteration's incremental bound still starts from the last
    # dense one, across the model change of the sparse iterations
    from paper_1409_4256_gb300 import emc
    torch, p = torch_cuda, small_problem
    nd, nrot, M = p["K"].shape[0], p["quat"].shape[0], 64
    a = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision="bf16_split",
                    w_floor=p["w_floor"], store_scores=True, n_cand=M)
    d = emc.Context(p["N"], p["q"], p["quat"], p["w"], nd, precision="bf16_split",
                    w_floor=p["w_floor"], store_scores=True, dense_estep=True)
    for c in (a, d):
        c.set_frames(torch.as_tensor(p["K"], device="cuda"))
    rng = np.random.default_rng(3)
    a.set_candidates(torch.as_tensor(
        np.stack([rng.choice(nrot, M, replace=False) for _ in range(nd)]).astype(np.int32),
        device="cuda"))
    g = torch.as_tensor(p["grid"].astype(np.float32), device="cuda")
    g1, _ = a.iteration(g)
    g2, _ = _same_input_check(a, d, g1)
    g3, _ = a.sparse_iteration(g2)
    g4, _ = a.sparse_iteration(g3)
    _, s = _same_input_check(a, d, g4)
    assert s["pass1_delta"] == 1
