"""GPU R-hat_max benchmark (Section 4.2; Algorithm A2's block shuffle)
against the oracle on the same accumulated draws and the same Philox picks
(FP64 on both sides: rtol 1e-9)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("D, n", [(5, 400), (3, 350), (1, 100)])   # 350/25 = 14 batches: uneven blocks
def test_shuffle_matches_oracle(torch, orc, D, n):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks(N=203, p=5, K=15, L=5)
    b = 25
    pc = PCV.from_workload(w, batch_size=b)
    pc.set_positions(np.zeros((w.n_chains, w.dim)), step_size=0.01)
    s = W.random_shat_series(w.n_chains, n, rho=0.6, loc=-40.0, scale=2.0, seed=31)
    s[3] += 1.5                                   # one chain off, so folds differ
    pc.accumulate(torch.tensor(s, device="cuda"))
    R = 300
    mx, allv = pc.rhat_shuffle(D, R, per_fold=True)
    omx, oall = orc.shuffle_series(s, L=w.chains_per_fold, b=b, D=D, R=R, seed=w.seed)
    np.testing.assert_allclose(allv, oall, rtol=1e-9)
    np.testing.assert_allclose(mx, omx, rtol=1e-9)
    pc.close()


def test_shuffle_on_a_run_and_errors(torch):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_BAD_STATE, E_INVALID_ARG
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    pc = PCV.from_workload(w, batch_size=10)
    pc.warmup(60, 30)
    with pytest.raises(PCVError) as e:
        pc.rhat_shuffle(5, 10)
    assert e.value.status == E_BAD_STATE
    pc.sample(200)
    with pytest.raises(PCVError) as e:
        pc.rhat_shuffle(21, 10)                   # 20 batches < 21 blocks
    assert e.value.status == E_INVALID_ARG
    mx = pc.rhat_shuffle(5, 500)
    assert np.all(np.isfinite(mx)) and mx.min() > 0.99
    # the run has mixed: its R-hat_max sits inside the benchmark's range
    assert pc.diagnostics()["rhat_max"] <= mx.max() * 1.02
    pc.close()
