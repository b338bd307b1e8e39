"""Pins for the covariate-selection mask (Appendix B's M_j) and the pairwise
comparison of two models on the same folds (eq. sel-cv, norm-approx,
mc-var), through the conjugate Gaussian closed form."""
import dataclasses

import numpy as np
from scipy import stats

from paper_2310_07002_b300 import workloads as W


def closed_form_elpd(w, k, cols):
    """Exact joint held-out log density of fold k for the Gaussian linear
    model on the design columns `cols` (sigma known, beta ~ N(0, sd^2 I))."""
    train, test = w.fold != k, w.fold == k
    X = w.X[:, cols]
    s2 = w.sigma_known ** 2
    S = np.linalg.inv(X[train].T @ X[train] / s2 + np.eye(len(cols)) / w.beta_prior_sd ** 2)
    mu = S @ X[train].T @ w.y[train] / s2
    Xe = X[test]
    cov = s2 * np.eye(test.sum()) + Xe @ S @ Xe.T
    return stats.multivariate_normal(Xe @ mu, cov).logpdf(w.y[test])


def run(orc, w):
    prob = orc.problem_from_workload(w)
    r = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=w.step_size, b=w.batch_size)
    r.fulldata(200, 250)
    r.fold_warmup(w.n_fold_warmup)
    r.sample(w.n_draws)
    fo, _ = r.results()
    return fo, r.state()


def test_masked_model_is_the_sub_design_model(orc):
    w = W.gauss_blocks()
    active = np.array([1, 0, 1, 1, 0], np.int32)
    wb = dataclasses.replace(w, active=active)
    fo, st = run(orc, wb)
    cols = np.nonzero(active)[0]
    assert np.all(st["theta"][:, active == 0] == 0.0)          # held at zero throughout
    for k in range(w.K):
        ref = closed_form_elpd(w, k, cols)
        assert abs(fo["elpd"][k] - ref) < 4 * fo["mcse"][k], (k, fo["elpd"][k], ref)


def test_pairwise_comparison(orc):
    w = W.gauss_blocks()
    active = np.array([1, 1, 1, 0, 1], np.int32)
    fa, _ = run(orc, w)
    fb, _ = run(orc, dataclasses.replace(w, active=active))
    c = orc.compare(fa["elpd"], fa["mcse"], fb["elpd"], fb["mcse"])
    # per-fold differences against the closed forms of both models
    full, sub = np.arange(w.p), np.nonzero(active)[0]
    dk_ref = np.array([closed_form_elpd(w, k, full) - closed_form_elpd(w, k, sub) for k in range(w.K)])
    assert np.all(np.abs(c["delta_k"] - dk_ref) < 4 * c["mcse_k"])
    assert abs(c["delta"] - (fa["elpd"].sum() - fb["elpd"].sum())) < 1e-9
    assert abs(c["se"] - np.sqrt(w.K * np.var(c["delta_k"], ddof=1))) < 1e-9
    assert abs(c["prob"] - stats.norm.cdf(c["delta"] / c["se"])) < 1e-12
    assert abs(c["mcse"] - np.sqrt((fa["mcse"] ** 2).sum() + (fb["mcse"] ** 2).sum())) < 1e-12
    # swapping the models negates the difference and complements the probability
    r = orc.compare(fb["elpd"], fb["mcse"], fa["elpd"], fa["mcse"])
    assert abs(r["delta"] + c["delta"]) < 1e-12 and abs(r["prob"] + c["prob"] - 1.0) < 1e-12


def test_chain_base_replays_the_chains_of_a_longer_run(orc):
    # one fold, so that chain ids and folds do not interact: a run of L0
    # chains with chain_base = L0 is chains L0 .. 2 L0 - 1 of a run of 2 L0
    # chains (the same Philox ids), bit for bit, from the pool start index
    # on (Appendix B's two-model runs replay model B's chains this way)
    w = W.gauss_blocks()
    fold = np.where(np.arange(w.N) < 20, 0, -1).astype(np.int32)
    w1 = dataclasses.replace(w, fold=fold, K=1)
    prob = orc.problem_from_workload(w1)
    L0 = 3
    long = orc.OraclePCV(prob, 2 * L0, w.seed, w.leapfrog_steps, eps=0.05, b=5)
    short = orc.OraclePCV(prob, L0, w.seed, w.leapfrog_steps, eps=0.05, b=5, chain_base=L0)
    for r in (long, short):
        r.fulldata(0, 40)
        r.fold_warmup(0)
    np.testing.assert_array_equal(short.state()["theta"], long.state()["theta"][L0:])
    for r in (long, short):
        r.sample(10)
    a, b = long.state(), short.state()
    np.testing.assert_array_equal(b["theta"], a["theta"][L0:])
    np.testing.assert_array_equal(b["shat"], a["shat"][L0:])
    # and base 0 is not base L0: the first chains of the long run differ
    assert not np.array_equal(b["theta"], a["theta"][:L0])
