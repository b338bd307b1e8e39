"""Pins for the oracle's Hyvarinen (Algorithm A3) and Dawid-Sebastiani
(Algorithm A4) scores on the conjugate Gaussian linear model, whose fold
predictives are Gaussian with closed-form mean and covariance:
  m = X_te mu_k, S = sigma^2 I + X_te Sigma_k X_te'
  DSS_k = -log|S| - (y - m)' S^-1 (y - m)
  HS_k  = sum_i [2 / sigma^2 - ((y_i - m_i)^2 + 2 x_i' Sigma_k x_i) / sigma^4]
(HS per test observation, positively oriented)."""
import numpy as np

from paper_2310_07002_b300 import workloads as W
from tests.test_oracle_conjugate import closed_form


def exact_scores(w, k):
    mu, S, _ = closed_form(w, k)
    test = w.fold == k
    Xe, ye = w.X[test], w.y[test]
    s2 = w.sigma_known ** 2
    m = Xe @ mu
    v = np.einsum("ij,jk,ik->i", Xe, S, Xe)
    cov = s2 * np.eye(test.sum()) + Xe @ S @ Xe.T
    sign, ld = np.linalg.slogdet(cov)
    r = ye - m
    q = r @ np.linalg.solve(cov, r)
    dss = -ld - q
    hs = np.sum(2.0 / s2 - (r ** 2 + 2.0 * v) / s2 ** 2)
    return hs, dss, q


def test_hs_and_dss_match_the_closed_forms(orc):
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=w.step_size, b=w.batch_size)
    run.enable_extra_scores(3)
    run.fulldata(200, 250)
    run.fold_warmup(w.n_fold_warmup)
    n_draws = 3000
    run.sample(n_draws)
    hs, dss = run.extra_scores()
    n = w.chains_per_fold * n_draws
    for k in range(w.K):
        h_ref, d_ref, q = exact_scores(w, k)
        # HS varies with theta only through the small posterior spread of the
        # predictive mean: within 1 %
        assert abs(hs[k] - h_ref) < 0.01 * abs(h_ref), (k, hs[k], h_ref)
        # DSS estimates a T x T covariance from n nearly independent
        # predictive draws: the quadratic form q has relative noise
        # sqrt(2 / n), log|S| noise sqrt(2 T / n) and bias ~ T (T + 1) / (2 n)
        T = int((w.fold == k).sum())
        sd = np.sqrt(2.0 * q * q / n + 2.0 * T / n)
        assert abs(dss[k] - d_ref) < 4.0 * sd + T * (T + 1) / n, (k, dss[k], d_ref, sd)


def blocks_of(w, K, T):
    """The workload's first K * T rows as K folds of T consecutive rows."""
    import dataclasses
    fold = np.full(w.N, -1, np.int32)
    fold[:K * T] = np.arange(K * T) // T
    return dataclasses.replace(w, fold=fold, K=K)


def test_logistic_dss_at_a_fixed_position(orc):
    # Chains held at one position (a step size far below the positions'
    # resolution): every draw's predictive is Bernoulli(p_i), p_i =
    # sigmoid(x_i' theta), independent across the test rows, so the DSS
    # (Algorithm A4, with the sample mean and covariance of the draws) tends
    # to -sum log p_i (1 - p_i) - sum (y_i - p_i)^2 / (p_i (1 - p_i)).  The
    # estimator's own spread at this draw count is measured by simulating it
    # with numpy's generator (brute force).
    w = blocks_of(W.logistic_loo(N=200, p=3, L=4), K=5, T=3)
    prob = orc.problem_from_workload(w)
    th0 = np.tile(w.truth["beta"], (w.n_chains, 1))
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=1e-12, b=50)
    run.enable_extra_scores(2)
    run.set_state(th0, eps=1e-12)
    n_draws = 2000
    run.sample(n_draws)
    hs, dss = run.extra_scores()
    assert np.all(np.isnan(hs))                          # no HS for a discrete response
    assert np.allclose(run.state()["theta"], th0, rtol=0, atol=1e-6)
    n = w.chains_per_fold * n_draws
    rng = np.random.default_rng(3)
    for k in range(w.K):
        rows = np.where(w.fold == k)[0]
        pk = 1.0 / (1.0 + np.exp(-(w.X[rows] @ w.truth["beta"])))
        yk = w.y[rows]
        exact = -np.sum(np.log(pk * (1 - pk))) - np.sum((yk - pk) ** 2 / (pk * (1 - pk)))

        def estimate(d):
            mu = d.mean(axis=0)
            S = np.cov(d, rowvar=False, ddof=1)
            r = yk - mu
            return -np.linalg.slogdet(S)[1] - r @ np.linalg.solve(S, r)

        sims = [estimate((rng.random((n, 3)) < pk).astype(float)) for _ in range(200)]
        sd = np.std(sims)
        assert abs(np.mean(sims) - exact) < 0.2 * sd + 0.05 * abs(exact)   # the simulation agrees with the limit
        assert abs(dss[k] - exact) < 5 * sd + abs(np.mean(sims) - exact), (k, dss[k], exact, sd)


def test_logistic_dss_equals_two_pass_on_the_same_draws(orc):
    # The predictive draws are reproducible: with the chains held at theta,
    # ytil_i = 1 iff u_i < sigmoid(x_i' theta), u_i from word i % 4 of the
    # Philox block (i / 4, chain, iteration, stream 5) -- the generator is
    # pinned by its known-answer vectors.  The DSS from the online sums must
    # equal the two-pass sample mean and covariance (n - 1 dof) of those draws.
    w = blocks_of(W.logistic_loo(N=200, p=3, L=4), K=5, T=3)
    prob = orc.problem_from_workload(w)
    th0 = np.tile(w.truth["beta"], (w.n_chains, 1))
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=1e-12, b=50)
    run.enable_extra_scores(2)
    run.set_state(th0, eps=1e-12)
    n_draws = 50
    run.sample(n_draws)
    _, dss = run.extra_scores()
    key = [w.seed & 0xFFFFFFFF, w.seed >> 32]
    for k in range(w.K):
        rows = np.where(w.fold == k)[0]
        pk = 1.0 / (1.0 + np.exp(-(w.X[rows] @ w.truth["beta"])))
        d = []
        for l in range(w.chains_per_fold):
            c = k * w.chains_per_fold + l
            for it in range(n_draws):
                words = orc.philox([0, c, it, 5], key)
                u = (np.array(words[:3], dtype=np.float64) + 0.5) / 2.0 ** 32
                d.append((u < pk).astype(float))
        d = np.array(d)
        mu = d.mean(axis=0)
        S = np.cov(d, rowvar=False, ddof=1)
        r = w.y[rows] - mu
        ref = -np.linalg.slogdet(S)[1] - r @ np.linalg.solve(S, r)
        assert abs(dss[k] - ref) <= 1e-9 * max(1.0, abs(ref)), (k, dss[k], ref)
