"""Closed-form pin of a whole oracle PCV run on the conjugate Gaussian
linear model (sigma known, beta ~ N(0, 10^2 I), K = 10 contiguous blocks).

Fold posterior: beta | y_train ~ N(mu_k, S_k), S_k = (X'X/s^2 + I/100)^-1,
mu_k = S_k X'y / s^2.  Exact joint held-out log predictive:
log N(y_test | X_test mu_k, s^2 I + X_test S_k X_test').  Every fold's elpd
and every posterior mean must fall within 4 MCSE of the closed form."""
import numpy as np
from scipy import stats

from paper_2310_07002_b300 import workloads as W


def closed_form(w, k):
    train, test = w.fold != k, w.fold == k
    Xt, yt = w.X[train], w.y[train]
    s2 = w.sigma_known ** 2
    S = np.linalg.inv(Xt.T @ Xt / s2 + np.eye(w.p) / w.beta_prior_sd ** 2)
    mu = S @ Xt.T @ yt / s2
    Xe = w.X[test]
    cov = s2 * np.eye(test.sum()) + Xe @ S @ Xe.T
    elpd = stats.multivariate_normal(Xe @ mu, cov).logpdf(w.y[test])
    return mu, S, elpd


import pytest


@pytest.mark.parametrize("eps, jitter", [(0.05, -1.0),   # the config: fixed step, no jitter
                                         (0.05, 0.5),    # jittered step size
                                         (-1.0, -1.0)])  # adapted: mass windows, cap, jitter
def test_conjugate_fold_posteriors_and_elpd(orc, eps, jitter):
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    L, b = w.chains_per_fold, w.batch_size
    run = orc.OraclePCV(prob, L, w.seed, w.leapfrog_steps, eps=eps, b=b, jitter=jitter)
    run.fulldata(200, 250)
    run.fold_warmup(w.n_fold_warmup)
    run.sample(w.n_draws)
    fo, to = run.results()
    mean, bmean, bM2 = run.theta_stats()
    n, a = w.n_draws, w.n_draws // b
    for k in range(w.K):
        mu, S, elpd = closed_form(w, k)
        assert abs(fo["elpd"][k] - elpd) < 4 * fo["mcse"][k], (k, fo["elpd"][k], elpd)
        sl = slice(k * L, (k + 1) * L)
        # pooled batch-means variance of the posterior mean (eq. bmvar)
        pm = mean[sl].mean(axis=0)
        ss = bM2[sl].sum(axis=0) + a * ((bmean[sl] - pm) ** 2).sum(axis=0)
        mcse = np.sqrt(b * ss / (L * a - 1) / (L * n))
        assert np.all(np.abs(pm - mu) < 4 * mcse), (k, pm, mu, mcse)
        # posterior sd in the right range as a sanity check of mixing
    assert to["rhat_max"] < 1.05
    assert fo["accept_rate"].min() > 0.5
