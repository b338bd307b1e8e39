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
