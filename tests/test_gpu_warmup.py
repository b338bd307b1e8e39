"""GPU parity of the full-data warm-up (warm-up reuse, Section 3.1) and of the
fold-chain starts (Algorithm 1) against the FP64 oracle, through the C ABI.

* The adaptation arithmetic (dual averaging of the step size, Hoffman &
  Gelman 2014, and the two diagonal-mass windows): the GPU's adaptation
  kernel and the oracle's adaptation driven by the same acceptance
  statistics and positions (pcv_adapt_trace / oracle.adapt_trace): step size
  and inverse mass after every iteration within 1e-6 relative (the GPU keeps
  them in FP32; its dual-averaging state is FP64).  A whole warm-up cannot be
  compared path by path: while dual averaging probes step sizes far beyond
  the stable range, leapfrog trajectories amplify FP32 rounding and the GPU
  and oracle chains part; so:
* the whole GPU warm-up is checked against what the mathematics fixes: on the
  conjugate Gaussian model its adapted inverse mass equals the exact
  full-data posterior variances within the windows' sampling error (the same
  pin as the oracle's);
* each fold chain's start is bit for bit the pool draw at the index
  floor(w0 n_pool / 2^32) (w0 from Philox stream 2) that the oracle computes
  (integer work: exact).
"""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu

ST_INIT = 2


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def _inputs(n, d, seed):
    rng = np.random.default_rng(seed)
    acc = rng.uniform(0.2, 1.0, (n, 4))
    # spread growing with the iteration: a window off by one iteration would
    # change the variances far beyond the tolerance
    scale = (1.0 + np.arange(n)) ** 1.5
    draws = (rng.standard_normal((n, 4, d)) * scale[:, None, None] + 3.0).astype(np.float32)
    return acc, draws


@pytest.mark.parametrize("n,adapt_mass", [(64, True), (200, True), (37, True), (50, False)])
def test_adaptation_kernel_matches_oracle(torch, orc, n, adapt_mass):
    from paper_2310_07002_b300.pcv import PCV
    w = W.ar2_hvblock(T=300, K=5, L=2)            # dim 3: two lags and log sigma
    pc = PCV.from_workload(w)
    acc, draws = _inputs(n, w.dim, 17 + n)
    eps_g, minv_g, fin_g = pc.adapt_trace(acc, draws, eps0=0.1, adapt_mass=adapt_mass)
    # the oracle takes the chains' mean acceptance statistic (summed in chain order)
    mean_acc = ((acc[:, 0] + acc[:, 1]) + acc[:, 2] + acc[:, 3]) / 4
    eps_o, minv_o, fin_o = orc.adapt_trace(mean_acc, draws.astype(np.float64), eps0=0.1, adapt_eps=True,
                                           adapt_mass=adapt_mass)
    np.testing.assert_allclose(eps_g, eps_o, rtol=1e-6)
    np.testing.assert_allclose(minv_g, minv_o, rtol=1e-6)
    assert abs(fin_g / fin_o - 1) < 1e-6
    if adapt_mass:
        assert np.abs(minv_o[-1] - 1.0).max() > 1.0         # the windows did act
    # the context is left as it was: a warm-up afterwards runs normally
    pc.warmup(20, 10)
    pc.close()


def test_adaptation_kernel_keeps_masked_covariates_at_zero(torch, orc):
    import dataclasses
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks(N=80, p=4, K=4, L=2)
    act = np.array([1, 0, 1, 1], np.int32)
    w = dataclasses.replace(w, active=act)
    pc = PCV.from_workload(w)
    acc, draws = _inputs(48, w.dim, 5)
    draws[:, :, 1] = 0.0                         # held coordinates stay at 0
    eps_g, minv_g, _ = pc.adapt_trace(acc, draws, eps0=0.1)
    mean_acc = ((acc[:, 0] + acc[:, 1]) + acc[:, 2] + acc[:, 3]) / 4
    m0 = np.array([1.0, 0.0, 1.0, 1.0])
    eps_o, minv_o, _ = orc.adapt_trace(mean_acc, draws.astype(np.float64), eps0=0.1, minv0=m0, active=act)
    assert np.all(minv_g[:, 1] == 0.0)
    np.testing.assert_allclose(minv_g, minv_o, rtol=1e-6)
    np.testing.assert_allclose(eps_g, eps_o, rtol=1e-6)
    pc.close()


def test_fold_starts_are_the_indexed_pool_draws(torch, orc):
    from paper_2310_07002_b300.pcv import PCV
    for w, first_fold in ((W.gauss_blocks(), 0), (W.logistic_loo(N=400, p=6, K=20, L=4), 7)):
        pc = PCV.from_workload(w, step_size=-1.0, n_fulldata_draws=250, first_fold=first_fold)
        pc.warmup(100, 0)
        th, _, _ = pc.positions()
        pool = pc.pool()
        n_pool = pool.shape[0]
        assert n_pool == 1000
        L = w.chains_per_fold
        idx = np.array([orc.index(w.seed, first_fold * L + c, 0, ST_INIT, n_pool) for c in range(pc.C)])
        np.testing.assert_array_equal(th, pool[idx])
        # the pool holds distinct draws, so the check pins the index
        assert len({tuple(r) for r in pool[idx]}) > 0.9 * len(set(idx.tolist()))
        pc.close()


@pytest.mark.parametrize("seed", [11, 12])
def test_gpu_warmup_inverse_mass_matches_conjugate_posterior(torch, seed):
    # conjugate Gaussian linear model: the full-data posterior variances are
    # diag (X'X + I / 100)^-1; the second window (3 n / 8 iterations x 4
    # chains) estimates them to sqrt(2 / m), shrunk as m / (m + 5)
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    n = 2000
    pc = PCV.from_workload(w, step_size=-1.0, seed=seed)
    pc.warmup(n, 0)
    eps, minv = pc.adaptation()
    pc.close()
    X = w.X.astype(np.float64)
    var = np.diag(np.linalg.inv(X.T @ X / w.sigma_known ** 2 + np.eye(w.p) / w.beta_prior_sd ** 2))
    m = 4 * ((7 * n) // 8 - n // 2)
    wgt = m / (m + 5.0)
    rel = minv / (wgt * var + 1e-3 * (1 - wgt)) - 1.0
    sd = np.sqrt(2.0 / m)
    assert np.all(np.abs(rel) < 4 * sd), (rel, sd)
    assert abs(eps - np.pi / 2 / w.leapfrog_steps) < 1e-6       # capped at pi/2 / L_f
