"""Pins for the oracle's fold-masked log density, gradient and held-out log
predictive (eq. mask-log-prob / mask-log-pred, Appendix B).

Independent routes: Gaussian sufficient statistics (X'X, X'y), scipy's
log densities summed over masks built here from the definitions, and
central finite differences of the oracle's own log density."""
import numpy as np
import pytest
from scipy import special, stats

from paper_2310_07002_b300 import workloads as W


def masks(fold, k, h=0):
    """Appendix B masks from the definition: test = fold == k, train = fold != k,
    minus h rows either side of the (contiguous) test block."""
    fold = np.asarray(fold)
    test = fold == k
    train = fold != k
    if h > 0 and test.any():
        idx = np.nonzero(test)[0]
        lo, hi = idx.min() - h, idx.max() + h
        n = np.arange(fold.size)
        train &= ~((n >= lo) & (n <= hi))
    return train, test


def fd_grad(f, x, rel=1e-6):
    g = np.empty_like(x)
    for j in range(x.size):
        hstep = rel * max(1.0, abs(x[j]))
        xp = x.copy(); xp[j] += hstep
        xm = x.copy(); xm[j] -= hstep
        g[j] = (f(xp) - f(xm)) / (2 * hstep)
    return g


def test_gauss_known_sigma_sufficient_stats(orc):
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    th = W.random_theta(w.dim, 3, scale=1.0, seed=3)
    s2 = w.sigma_known ** 2
    for k in [0, 4, 9, -1]:
        train, test = masks(w.fold, k) if k >= 0 else (np.ones(w.N, bool), np.zeros(w.N, bool))
        Xt, yt = w.X[train], w.y[train]
        XtX, Xty, yty = Xt.T @ Xt, Xt.T @ yt, yt @ yt
        n = train.sum()
        for beta in th:
            lp, g, sh = orc.log_density(prob, k, beta)
            quad = yty - 2 * beta @ Xty + beta @ XtX @ beta
            lp_ref = (-0.5 * n * np.log(2 * np.pi * s2) - 0.5 * quad / s2
                      + stats.norm.logpdf(beta, 0, w.beta_prior_sd).sum())
            g_ref = (Xty - XtX @ beta) / s2 - beta / w.beta_prior_sd ** 2
            sh_ref = stats.norm.logpdf(w.y[test], w.X[test] @ beta, w.sigma_known).sum()
            assert abs(lp - lp_ref) < 1e-9 * max(1, abs(lp_ref))
            assert np.allclose(g, g_ref, rtol=1e-10, atol=1e-9)
            assert abs(sh - sh_ref) < 1e-9 * max(1, abs(sh_ref))


def test_logistic_against_scipy_and_fd(orc):
    w = W.logistic_loo(N=300, p=6, K=40, L=2)
    prob = orc.problem_from_workload(w)
    for k in [0, 39, -1]:
        train, test = masks(w.fold, k) if k >= 0 else (np.ones(w.N, bool), np.zeros(w.N, bool))
        for beta in W.random_theta(w.dim, 2, seed=5):
            lp, g, sh = orc.log_density(prob, k, beta)
            eta = w.X @ beta
            ll = w.y * special.log_expit(eta) + (1 - w.y) * special.log_expit(-eta)
            lp_ref = ll[train].sum() + stats.norm.logpdf(beta, 0, w.beta_prior_sd).sum()
            assert abs(lp - lp_ref) < 1e-10 * max(1, abs(lp_ref))
            assert abs(sh - ll[test].sum()) < 1e-10
            gfd = fd_grad(lambda b: orc.log_density(prob, k, b)[0], beta)
            assert np.allclose(g, gfd, rtol=1e-6, atol=1e-6)


def test_ar_hvblock_masks_and_fd(orc):
    w = W.ar2_hvblock(T=400, K=15)
    prob = orc.problem_from_workload(w)
    assert w.dim == 3
    for k in [0, 7, 14]:
        train, test = masks(w.fold, k, w.hv_buffer)
        # the buffer removes exactly h rows either side (interior folds)
        assert test.sum() == 10
        for th in W.random_theta(3, 2, scale=0.4, seed=9):
            lp, g, sh = orc.log_density(prob, k, th)
            sig = np.exp(th[2])
            ll = stats.norm.logpdf(w.y, w.X @ th[:2], sig)
            prior = (stats.norm.logpdf(th[:2], 0, 1).sum()
                     + stats.halfnorm.logpdf(sig, scale=w.sigma_prior_sd) + th[2])
            assert abs(lp - (ll[train].sum() + prior)) < 1e-9 * abs(lp)
            assert abs(sh - ll[test].sum()) < 1e-10 * max(1, abs(sh))
            gfd = fd_grad(lambda t: orc.log_density(prob, k, t)[0], th)
            assert np.allclose(g, gfd, rtol=1e-6, atol=1e-5)
    # interior fold: the train set drops the test block plus h = 10 rows each side
    train, _ = masks(w.fold, 7, w.hv_buffer)
    assert (~train).sum() == 10 + 2 * 10


def test_hier_against_scipy_and_fd(orc):
    w = W.hier_logo(G=8, p=3, L=2, mean_extra=6.0)
    prob = orc.problem_from_workload(w)
    d = w.dim
    assert d == 3 + 8 + 2
    for k in [0, 5, -1]:
        train, test = masks(w.fold, k) if k >= 0 else (np.ones(w.N, bool), np.zeros(w.N, bool))
        for th in W.random_theta(d, 2, scale=0.5, seed=13):
            lp, g, sh = orc.log_density(prob, k, th)
            beta, z, lt, ls = th[:3], th[3:11], th[11], th[12]
            tau, sig = np.exp(lt), np.exp(ls)
            ll = stats.norm.logpdf(w.y, w.X @ beta + tau * z[w.group], sig)
            prior = (stats.norm.logpdf(beta, 0, 1).sum() + stats.norm.logpdf(z).sum()
                     + stats.halfnorm.logpdf(tau, scale=1.0) + lt
                     + stats.halfnorm.logpdf(sig, scale=1.0) + ls)
            assert abs(lp - (ll[train].sum() + prior)) < 1e-9 * abs(lp)
            # LOGO: the held-out group is a new group; its rows are scored by
            # the group-level predictive (eq. group-marg) with the intercept
            # tau z integrated over z ~ N(0, 1): a multivariate normal with
            # covariance sigma^2 I + tau^2 11'
            ref = 0.0
            for grp in np.unique(w.group[test]):
                rows = test & (w.group == grp)
                m = int(rows.sum())
                cov = sig ** 2 * np.eye(m) + tau ** 2 * np.ones((m, m))
                ref += stats.multivariate_normal.logpdf(w.y[rows], w.X[rows] @ beta, cov)
            assert abs(sh - ref) < 1e-9 * max(1, abs(sh))
            gfd = fd_grad(lambda t: orc.log_density(prob, k, t)[0], th)
            assert np.allclose(g, gfd, rtol=1e-6, atol=1e-5)


def test_hier_heldout_group_is_integrated_over_its_intercept(orc):
    # the same quantity by numerical integration of the definition:
    # log int prod_n N(y_n | x_n beta + tau z, sigma^2) N(z | 0, 1) dz
    from scipy import integrate
    w = W.hier_logo(G=6, p=2, L=2, mean_extra=3.0)
    prob = orc.problem_from_workload(w)
    th = W.random_theta(w.dim, 1, scale=0.4, seed=5)[0]
    beta, lt, ls = th[:2], th[2 + 6], th[3 + 6]
    tau, sig = np.exp(lt), np.exp(ls)
    k = 3
    _, _, sh = orc.log_density(prob, k, th)
    rows = w.fold == k
    e = w.y[rows] - w.X[rows] @ beta
    c = np.max(stats.norm.logpdf(e, 0.0, sig).sum() + 0.0)   # scale for the integrand

    def integrand(z):
        return np.exp(stats.norm.logpdf(e, tau * z, sig).sum() - c) * stats.norm.pdf(z)
    val, _ = integrate.quad(integrand, -12, 12, epsabs=0, epsrel=1e-12, limit=400)
    assert abs(sh - (np.log(val) + c)) < 1e-8 * max(1.0, abs(sh))


def test_rows_in_no_test_set_always_train(orc):
    # logistic LOO with K < N: rows with fold -1 are in every training set
    w = W.logistic_loo(N=50, p=3, K=5, L=2)
    prob = orc.problem_from_workload(w)
    beta = np.array([0.3, -0.2, 0.1])
    lp_full, _, _ = orc.log_density(prob, -1, beta)
    eta = w.X @ beta
    ll = w.y * special.log_expit(eta) + (1 - w.y) * special.log_expit(-eta)
    for k in range(5):
        lp, _, sh = orc.log_density(prob, k, beta)
        assert abs((lp_full - lp) - ll[k]) < 1e-10
        assert abs(sh - ll[k]) < 1e-12
