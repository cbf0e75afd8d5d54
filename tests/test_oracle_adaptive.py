"""Pins of the adaptive schedule's oracle (Sec. 3.4, Eq. 3.1)."""
import numpy as np
from scipy.special import gammaln
from scipy.stats import poisson


def test_log_factorial_constant():
    from oracle import adaptive
    assert np.isclose(adaptive.log_factorial_constant([[0, 1, 2, 3]]), np.log(12.0), atol=1e-14)
    K = np.random.default_rng(20).poisson(3.0, size=(17, 29))
    assert np.isclose(adaptive.log_factorial_constant(K), gammaln(K + 1.0).sum(), rtol=1e-13)


def test_loglik_is_the_mixture_likelihood(oracle):
    # brute force: L = sum_k log sum_j w_j prod_i pmf(K_ik; W_ij)
    from oracle import adaptive
    rng = np.random.default_rng(21)
    W = rng.uniform(0.3, 3.0, size=(4, 6))
    w = rng.uniform(0.5, 1.5, size=4)
    w /= w.sum()
    K = rng.poisson(1.2, size=(5, 6))
    _, _, tot = oracle.estep(oracle.scores(W, w, K.astype(float)))
    lik = np.array([[w[j] * np.prod(poisson.pmf(K[k], W[j])) for j in range(4)] for k in range(5)])
    assert np.isclose(adaptive.log_likelihood(tot, K), np.log(lik.sum(1)).sum(), rtol=0, atol=1e-10)


def test_refinement_rule():
    from oracle import adaptive
    r = adaptive.should_refine
    assert not r(-1000.0, None)
    assert r(-1000.0, -1009.9)        # |dL| = 9.9 <= 10
    assert r(-1000.0, -990.0)         # a decrease of 1% also counts
    assert not r(-1000.0, -1010.05)  # 10.05 > 1% of |L^n| (but < 1% of |L^{n-1}|)
    assert r(-1000.0, -1000.0)
    assert r(-500.0, -520.0, threshold=0.05) and not r(-500.0, -530.0, threshold=0.05)
    assert r(200.0, 201.9) and not r(200.0, 202.1)  # |L| when L is positive


def test_schedule_follows_rule(oracle, small_problem):
    # a few iterations from d = 1; every refinement happens exactly where Eq. 3.1 holds
    from oracle import adaptive
    p = small_problem
    K = p["K"][:120]
    grid, hist = adaptive.run(p["grid"], p["q"], K, 1, 3, 6, p["w_floor"], threshold=0.01)
    ds = [h[0] for h in hist]
    assert ds[0] == 1 and all(b - a in (0, 1) for a, b in zip(ds, ds[1:])) and max(ds) <= 3
    assert [h[1] for h in hist] == [10 * (5 * d ** 3 + d) for d in ds]
    prev = None
    for (d, _, L), nxt in zip(hist, ds[1:] + [None]):
        want = adaptive.should_refine(L, prev, 0.01) and d < 3
        if nxt is not None:
            assert (nxt == d + 1) == want
        prev = None if want else L
    assert max(ds) > 1  # the synthetic start is close to the truth: the likelihood settles fast
    assert np.all(np.isfinite(grid)) and grid.min() >= 0
