"""Pins of the oracle's full-data warm-up adaptation (warm-up reuse,
Section 3.1): Nesterov dual averaging of the step size (Hoffman & Gelman
2014, Section 3.2.1) and the two regularised diagonal-mass windows.

Each check compares the oracle with something other than itself:
  * the dual-averaging iterates against Hoffman & Gelman's closed form of
    the iterate (their eq. 6: x_{t+1} = mu - sqrt(t)/gamma * mean-ish sum of
    the errors), written as a sum rather than as the oracle's recursion;
  * the averaged iterate against its explicit weighted sum;
  * closed-loop convergence to the acceptance target on a known acceptance
    curve;
  * the mass windows against numpy's sample variance over exactly the
    iterations [n/4, n/2) and [n/2, 7n/8) of known draws (and the test shows
    that a window one iteration off would fail);
  * the adapted inverse mass of a whole HMC warm-up against the exact
    full-data posterior variances of the conjugate Gaussian model;
  * the mean acceptance statistic of the last dual-averaging phase against
    the target 0.8.
"""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

DELTA, GAMMA, T0, KAPPA = 0.8, 0.05, 10.0, 0.75


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def hg_closed_form(accept, eps0):
    """log step size after each of t = 1..n updates, and the averaged
    iterate, from the closed forms: x_t = mu - sqrt(t) / (gamma (t + t0))
    sum_{i<=t} (delta - a_i) with mu = log(10 eps0); xbar_t = sum_i
    eta_i x_i prod_{i<j<=t} (1 - eta_j), eta_i = i^-kappa."""
    n = len(accept)
    t = np.arange(1, n + 1, dtype=np.float64)
    mu = np.log(10.0 * eps0)
    x = mu - np.sqrt(t) / (GAMMA * (t + T0)) * np.cumsum(DELTA - np.asarray(accept))
    eta = t ** -KAPPA
    xbar = 0.0
    for i in range(n):
        xbar += eta[i] * x[i] * np.prod(1.0 - eta[i + 1:])
    return x, xbar


def test_dual_averaging_matches_closed_form(orc):
    rng = np.random.default_rng(5)
    n = 400
    acc = rng.uniform(0.0, 1.0, n)
    draws = np.zeros((n, 1, 2))
    eps, minv, fin = orc.adapt_trace(acc, draws, eps0=0.3, adapt_eps=True, adapt_mass=False)
    x, xbar = hg_closed_form(acc, 0.3)
    np.testing.assert_allclose(np.log(eps), x, rtol=0, atol=1e-10)
    assert abs(np.log(fin) - xbar) < 1e-10
    # no mass adaptation asked: the inverse mass stays as given
    assert np.all(minv == 1.0)


def test_dual_averaging_reaches_the_target_in_closed_loop(orc):
    # acceptance curve a(eps) = exp(-eps^2): the target 0.8 is met at
    # eps* = sqrt(-log 0.8); the oracle's updates, fed back through the
    # curve, must settle there (a sign, target or gain mistake does not)
    f = lambda e: np.exp(-e * e)
    eps_star = np.sqrt(-np.log(DELTA))
    n = 300
    acc = []
    e = 0.05
    for _ in range(n):
        acc.append(f(e))
        eps, _, fin = orc.adapt_trace(np.array(acc), np.zeros((len(acc), 1, 1)), eps0=0.05,
                                      adapt_eps=True, adapt_mass=False)
        e = eps[-1]
    assert abs(fin / eps_star - 1) < 0.01, (fin, eps_star)
    assert abs(np.mean(acc[-100:]) - DELTA) < 0.01


def test_mass_windows_use_exactly_the_two_windows(orc):
    n, nc, d = 64, 4, 3                       # windows [16, 32) and [32, 56)
    w0, w1, w2 = n // 4, n // 2, (7 * n) // 8
    rng = np.random.default_rng(11)
    # spread growing with the iteration, so that a window shifted by one
    # iteration changes the variance well beyond the tolerance
    scale = (1.0 + np.arange(n)) ** 1.5
    draws = rng.standard_normal((n, nc, d)) * scale[:, None, None] + 3.0
    acc = np.full(n, 0.9)
    minv0 = np.array([2.0, 3.0, 4.0])
    eps, minv, fin = orc.adapt_trace(acc, draws, eps0=0.1, adapt_eps=True, adapt_mass=True, minv0=minv0)

    def expected(lo, hi):
        v = draws[lo:hi].reshape(-1, d)
        m = v.shape[0]
        wgt = m / (m + 5.0)
        return wgt * v.var(axis=0, ddof=1) + 1e-3 * (1.0 - wgt)

    e1, e2 = expected(w0, w1), expected(w1, w2)
    # unchanged before the end of the first window
    assert np.all(minv[: w1 - 1] == minv0)
    np.testing.assert_allclose(minv[w1 - 1], e1, rtol=1e-12)
    assert np.all(minv[w1: w2 - 1] == minv[w1 - 1])
    np.testing.assert_allclose(minv[w2 - 1], e2, rtol=1e-12)
    assert np.all(minv[w2:] == minv[w2 - 1])
    # the check is sensitive to each bound: one iteration off fails it
    for lo, hi, ref in [(w0 - 1, w1, e1), (w0 + 1, w1, e1), (w0, w1 + 1, e1), (w0, w1 - 1, e1),
                        (w1 - 1, w2, e2), (w1 + 1, w2, e2), (w1, w2 + 1, e2), (w1, w2 - 1, e2)]:
        assert np.max(np.abs(expected(lo, hi) / ref - 1)) > 1e-3


def test_dual_averaging_restarts_from_the_current_step_after_each_window(orc):
    n, nc, d = 64, 4, 2
    w1, w2 = n // 2, (7 * n) // 8
    rng = np.random.default_rng(3)
    acc = rng.uniform(0.3, 1.0, n)
    draws = rng.standard_normal((n, nc, d))
    eps, _, fin = orc.adapt_trace(acc, draws, eps0=0.2, adapt_eps=True, adapt_mass=True)
    # before the first window ends: one dual-averaging run from eps0
    x, _ = hg_closed_form(acc[:w1], 0.2)
    np.testing.assert_allclose(np.log(eps[:w1]), x, atol=1e-10)
    # then restarts with mu = log(10 eps) at the step size in force
    x2, _ = hg_closed_form(acc[w1:w2], eps[w1 - 1])
    np.testing.assert_allclose(np.log(eps[w1:w2]), x2, atol=1e-10)
    x3, xbar3 = hg_closed_form(acc[w2:], eps[w2 - 1])
    np.testing.assert_allclose(np.log(eps[w2:]), x3, atol=1e-10)
    # the final step size averages only the last phase's iterates
    assert abs(np.log(fin) - xbar3) < 1e-10


def test_masked_covariates_keep_zero_inverse_mass(orc):
    n, nc, d = 40, 4, 4
    rng = np.random.default_rng(8)
    draws = rng.standard_normal((n, nc, d))
    active = np.array([1, 0, 1], np.int32)          # p = 3 covariates; coordinate 3 is not a covariate
    minv0 = np.array([1.0, 0.0, 1.0, 1.0])
    _, minv, _ = orc.adapt_trace(np.full(n, 0.8), draws, adapt_mass=True, minv0=minv0, active=active)
    assert np.all(minv[:, 1] == 0.0)
    assert np.all(minv[-1, [0, 2, 3]] > 0.1)


def conjugate_fulldata_variances(w):
    X = w.X.astype(np.float64)
    S = np.linalg.inv(X.T @ X / w.sigma_known ** 2 + np.eye(w.p) / w.beta_prior_sd ** 2)
    return np.diag(S)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_adapted_inverse_mass_matches_conjugate_posterior(orc, seed):
    # conjugate Gaussian linear model (N = 200, p = 5, sigma = 1 known): the
    # full-data posterior is N(mu, Sigma), Sigma = (X'X + I / 100)^-1, so the
    # second window's estimate (3 n / 8 iterations x 4 chains) must be
    # w Sigma_jj + 1e-3 (1 - w) up to its sampling error sqrt(2 / m)
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    n = 2000
    run = orc.OraclePCV(prob, w.chains_per_fold, seed, w.leapfrog_steps, eps=-1.0, b=50)
    run.fulldata(n, 10)
    minv = run.state()["minv"]
    m = 4 * ((7 * n) // 8 - n // 2)
    wgt = m / (m + 5.0)
    ref = wgt * conjugate_fulldata_variances(w) + 1e-3 * (1.0 - wgt)
    rel = minv / ref - 1.0
    sd = np.sqrt(2.0 / m)
    assert np.all(np.abs(rel) < 4 * sd), (rel, sd)
    assert abs(np.mean(rel)) < 4 * sd / np.sqrt(w.p)


def test_adaptation_meets_the_acceptance_target(orc):
    # the mean acceptance statistic over the last dual-averaging phase is
    # the quantity dual averaging drives to delta = 0.8 (its closed form
    # leaves an O(1/sqrt(t)) offset: 0.008 at t = 250); with the step cap
    # and jitter off, fresh iterations at the averaged step size accept at a
    # comparable rate, and with the cap the step is pi/2 / L_f
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    run = orc.OraclePCV(prob, w.chains_per_fold, 7, w.leapfrog_steps, eps=-1.0, b=50,
                        traj_len=0.0, jitter=0.0)
    run.fulldata(2000, 500)
    tail, keep = run.fulldata_accept()
    assert abs(tail - DELTA) < 0.02, tail
    assert 0.75 < keep < 0.95, keep
    capped = orc.OraclePCV(prob, w.chains_per_fold, 7, w.leapfrog_steps, eps=-1.0, b=50)
    capped.fulldata(2000, 10)
    assert abs(capped.state()["eps"] - np.pi / 2 / w.leapfrog_steps) < 1e-15
    assert run.state()["eps"] > capped.state()["eps"]
