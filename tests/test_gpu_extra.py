"""GPU Hyvarinen and Dawid-Sebastiani scores (Algorithms A3, A4): against the
conjugate closed form, and against the oracle on the same sampler paths."""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W
from tests.test_oracle_extra import exact_scores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def test_extra_scores_closed_form(torch):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    pc = PCV.from_workload(w, extra_scores=3)
    pc.warmup(200, w.n_fold_warmup)
    n_draws = 3000
    pc.sample(n_draws)
    ex = pc.scores_extra()
    n = w.chains_per_fold * n_draws
    for k in range(w.K):
        h_ref, d_ref, q = exact_scores(w, k)
        assert abs(ex["hs"][k] - h_ref) < 0.01 * abs(h_ref), (k, ex["hs"][k], h_ref)
        T = int((w.fold == k).sum())
        sd = np.sqrt(2.0 * q * q / n + 2.0 * T / n)
        assert abs(ex["dss"][k] - d_ref) < 4.0 * sd + T * (T + 1) / n, (k, ex["dss"][k], d_ref)
    assert abs(ex["hs_total"] - ex["hs"].sum()) < 1e-9 and abs(ex["dss_total"] - ex["dss"].sum()) < 1e-9
    pc.close()


def test_extra_scores_follow_oracle_paths(torch, orc):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks(N=203, p=5, K=15, L=5)
    prob = orc.problem_from_workload(w)
    th0 = W.random_theta(w.dim, w.n_chains, scale=0.5, seed=41).astype(np.float32).astype(np.float64)
    pc = PCV.from_workload(w, step_size=0.05, batch_size=10, acov_max_lag=5, extra_scores=3)
    pc.set_positions(th0, step_size=0.05)
    pc.sample(40)
    th_gpu, _, _ = pc.positions()
    ex = pc.scores_extra()
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=0.05, b=10, M=5)
    run.enable_extra_scores(3)
    run.set_state(th0, eps=0.05)
    run.sample(40)
    hs, dss = run.extra_scores()
    on = np.linalg.norm(th_gpu - run.state()["theta"], axis=1) < 1e-3 * np.linalg.norm(th_gpu, axis=1)
    folds = [k for k in range(w.K) if on[k * w.chains_per_fold:(k + 1) * w.chains_per_fold].all()]
    assert len(folds) >= w.K // 2, folds
    for k in folds:
        assert abs(ex["hs"][k] - hs[k]) <= 1e-4 * abs(hs[k]), (k, ex["hs"][k], hs[k])
        assert abs(ex["dss"][k] - dss[k]) <= 1e-3, (k, ex["dss"][k], dss[k])
    pc.close()


def test_extra_scores_need_a_gaussian_row_model(torch):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_UNSUPPORTED
    for w in (W.logistic_loo(N=300, p=5, K=10, L=2), W.hier_logo(G=10, p=3, L=2)):
        with pytest.raises(PCVError) as e:
            PCV.from_workload(w, extra_scores=1)
        assert e.value.status == E_UNSUPPORTED


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_logistic_dss_equals_oracle_at_a_fixed_position(torch, orc, precision):
    # Algorithm A4 for the logistic model: predictive draws are Bernoulli
    # with the Philox stream-5 uniforms; with the chains held at one position
    # (a step far below FP32 resolution) the GPU draws the oracle's draws, so
    # the DSS must agree to rounding, and no HS exists for a discrete y
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    from tests.test_oracle_extra import blocks_of
    w = blocks_of(W.logistic_loo(N=200, p=3, L=4), K=5, T=3)
    th0 = np.tile(w.truth["beta"], (w.n_chains, 1)).astype(np.float32).astype(np.float64)
    pc = PCV.from_workload(w, step_size=1e-12, extra_scores=2, precision=PRECISIONS[precision])
    pc.set_positions(th0, step_size=1e-12)
    pc.sample(200)
    ex = pc.scores_extra()
    assert np.array_equal(pc.positions()[0], th0)
    run = orc.OraclePCV(orc.problem_from_workload(w), w.chains_per_fold, w.seed, w.leapfrog_steps, eps=1e-12, b=50)
    run.enable_extra_scores(2)
    run.set_state(th0, eps=1e-12)
    run.sample(200)
    hs, dss = run.extra_scores()
    assert np.all(np.isnan(ex["hs"])) and np.all(np.isnan(hs))
    np.testing.assert_allclose(ex["dss"], dss, rtol=1e-9)
    pc.close()
