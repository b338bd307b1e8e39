"""Two models in one context (Appendix B: models evaluated in parallel by
their covariate-selection masks M_j): model A's and model B's chains in the
same launches, compared by pcv_compare_pair (eq. sel-cv, norm-approx,
mc-var), through the C ABI.

* Paths: model A's half follows an oracle run of model A, model B's half
  an oracle run of model B whose chain ids start at K L (oracle chain_base),
  on the same Philox streams, with B's inverse mass = A's restricted to B's
  covariates: 90 % of chains within 1e-3 after 20 iterations (FP32 and the
  BF16 tensor-core path, as test_sampling_follows_oracle_paths).
* The comparison equals its definition on the context's own fold scores
  (delta_k = elpd_A,k - elpd_B,k, mcse_k = sqrt(MCSE_A,k^2 + MCSE_B,k^2),
  out = {sum, sqrt(K var), sqrt(sum mcse^2), Phi(delta / se)}) to 1e-12.
* A whole run (warm-up reuse included): B's inactive coefficients are 0 in
  every B chain, and model A's half reproduces a one-model run of A within
  4 MCSE per fold.
* Config 3 (hierarchical, leave-one-group-out): dropping the covariate with
  the largest true coefficient gives Pr(A better than B) > 0.999.
"""
import dataclasses

import numpy as np
import pytest
from scipy import stats

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


MASK_B = np.array([1, 1, 0, 1, 0], np.int32)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pair_follows_two_oracle_runs(torch, orc, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.gauss_blocks(bf16=precision == "bf16")
    K, L = w.K, w.chains_per_fold
    KL = K * L
    th0 = W.random_theta(w.dim, 2 * KL, scale=0.5, seed=43).astype(np.float32).astype(np.float64)
    th0[KL:, MASK_B == 0] = 0.0
    minv = np.linspace(0.6, 1.4, w.dim)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], step_size=0.05, batch_size=10,
                           acov_max_lag=5, active_b=MASK_B)
    assert pc.K == 2 * K and pc.C == 2 * KL
    pc.set_positions(th0, step_size=0.05, inv_mass_diag=minv)
    pc.sample(20)
    th_gpu, _, _ = pc.positions()
    pc.close()
    assert np.all(th_gpu[KL:, MASK_B == 0] == 0.0)
    mv32 = minv.astype(np.float32).astype(np.float64)
    for half, mask, base in ((0, None, 0), (1, MASK_B, KL)):
        wm = w if mask is None else dataclasses.replace(w, active=mask)
        mvm = mv32 if mask is None else mv32 * mask
        run = orc.OraclePCV(orc.problem_from_workload(wm), L, w.seed, w.leapfrog_steps, eps=0.05, minv=mvm,
                            b=10, M=5, chain_base=base)
        run.set_state(th0[half * KL:(half + 1) * KL], eps=0.05, minv=mvm)
        run.sample(20)
        err = rel_vec(th_gpu[half * KL:(half + 1) * KL], run.state()["theta"])
        assert np.mean(err < 1e-3) >= 0.9, (precision, half, np.sort(err)[-8:])


def test_pair_comparison_matches_its_definition(torch):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    pc = PCV.from_workload(w, batch_size=10, active_b=MASK_B)
    pc.warmup(200, 50)
    pc.sample(200)
    sc = pc.scores()
    c = pc.compare_pair()
    pc.close()
    K = w.K
    ea, eb = sc["elpd"][:K], sc["elpd"][K:]
    ma, mb = sc["mcse"][:K], sc["mcse"][K:]
    np.testing.assert_allclose(c["delta_k"], ea - eb, rtol=0, atol=1e-12)
    np.testing.assert_allclose(c["mcse_k"], np.sqrt(ma ** 2 + mb ** 2), rtol=1e-12)
    assert abs(c["delta"] - (ea - eb).sum()) < 1e-9
    assert abs(c["se"] - np.sqrt(K * np.var(ea - eb, ddof=1))) < 1e-9
    assert abs(c["mcse"] - np.sqrt((ma ** 2 + mb ** 2).sum())) < 1e-12
    assert abs(c["prob"] - stats.norm.cdf(c["delta"] / c["se"])) < 1e-12


def test_pair_whole_run_model_a_half_and_held_coefficients(torch):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    KL = w.K * w.chains_per_fold
    pc = PCV.from_workload(w, batch_size=50, active_b=MASK_B)
    pc.warmup(500, 200)
    pc.sample(1000)
    th, _, _ = pc.positions()
    sp = pc.scores()
    pc.close()
    assert np.all(th[KL:, MASK_B == 0] == 0.0) and np.all(th[:KL, MASK_B == 0] != 0.0)
    one = PCV.from_workload(w, batch_size=50)
    one.warmup(500, 200)
    one.sample(1000)
    s1 = one.scores()
    one.close()
    K = w.K
    tol = 4 * np.sqrt(sp["mcse"][:K] ** 2 + s1["mcse"] ** 2)
    assert np.all(np.abs(sp["elpd"][:K] - s1["elpd"]) < tol), (sp["elpd"][:K] - s1["elpd"], tol)


def test_pair_config3_drops_the_strongest_covariate(torch):
    # hierarchical varying-intercept model, leave-one-group-out (config 3,
    # 100 groups); model B lacks the covariate with the largest |beta|
    from paper_2310_07002_b300.pcv import PCV
    w = W.hier_logo(L=4)
    j = int(np.argmax(np.abs(w.truth["beta"])))
    mb = np.ones(w.p, np.int32)
    mb[j] = 0
    pc = PCV.from_workload(w, batch_size=50, active_b=mb)
    pc.warmup(500, 200)
    pc.sample(500)
    c = pc.compare_pair()
    pc.close()
    assert c["delta"] > 0 and c["prob"] > 0.999, c
    assert c["mcse"] < 0.05 * c["delta"]
