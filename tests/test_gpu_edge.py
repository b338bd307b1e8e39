"""Edge and degenerate cases of the CUDA path against the FP64 oracle,
through the C ABI, for the FP32 and the BF16 (tcgen05) forms:
  - p = 1 (a single covariate);
  - fewer rows than one 128-row chunk and fewer chains than one tile;
  - rows in no test set (fold id -1) between the test blocks;
  - saturated linear predictors (|eta| ~ 40: tanh and softplus at their
    limits) and all-equal responses (y all 1);
  - a single fold (K = 1) sampled end to end;
  - a fold with no test rows is rejected (E_INVALID_ARG).
Tolerances as in test_gpu_parity (FP32) and test_gpu_bf16 (BF16)."""
import dataclasses

import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-5, 1e-5), "bf16": (1e-4, 1e-2)}     # (log density, gradient)


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def rel_scalar(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


def check_log_density(torch, orc, w, precision, th, label):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    prec = PRECISIONS[precision]
    pc = PCV.from_workload(w, precision=prec)
    prob = orc.problem_from_workload(w)
    n = th.shape[0]
    folds = np.arange(n) % (w.K + 1)
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    lp, g, sh = pc.log_density(tt, torch.tensor(folds, dtype=torch.int32, device="cuda"), prec)
    torch.cuda.synchronize()
    lp, g, sh = lp.cpu().numpy(), g.cpu().double().numpy(), sh.cpu().numpy()
    th64 = tt.cpu().double().numpy()
    ref = [orc.log_density(prob, -1 if k == w.K else int(k), th64[i]) for i, k in enumerate(folds)]
    lr = np.array([r[0] for r in ref]); gr = np.array([r[1] for r in ref]); sr = np.array([r[2] for r in ref])
    e = (rel_scalar(lp, lr).max(), rel_scalar(sh, sr).max(), rel_vec(g, gr).max())
    print("%s %s: logp %.2e shat %.2e grad %.2e" % (label, precision, *e))
    tol_lp, tol_g = TOL[precision]
    assert e[0] <= tol_lp and e[1] <= tol_lp and e[2] <= tol_g
    pc.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_single_covariate(torch, orc, precision):
    w = W.logistic_loo(N=301, p=1, K=30, L=3, bf16=True)
    check_log_density(torch, orc, w, precision, W.random_theta(w.dim, 70, scale=0.5, seed=41), "p=1")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_less_than_one_chunk_and_one_tile(torch, orc, precision):
    # 37 rows (one partial 128-row chunk), 5 folds x 4 chains = 20 chains
    w = W.logistic_loo(N=37, p=6, K=5, L=4, bf16=True)
    check_log_density(torch, orc, w, precision, W.random_theta(w.dim, 18, scale=0.5, seed=42), "N=37")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_rows_in_no_test_set(torch, orc, precision):
    # test blocks of 10 rows with 15 unassigned rows between them
    w = W.logistic_loo(N=1000, p=12, K=40, L=2, bf16=True)
    fold = np.full(w.N, -1, np.int32)
    for k in range(40):
        fold[25 * k: 25 * k + 10] = k
    w = dataclasses.replace(w, fold=fold)
    check_log_density(torch, orc, w, precision, W.random_theta(w.dim, 90, scale=0.4, seed=43), "fold -1 rows")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_saturated_predictors_and_constant_response(torch, orc, precision):
    # |eta| up to ~40 (sigmoid and softplus at their limits), all y = 1
    w = W.logistic_loo(N=500, p=8, K=20, L=2, bf16=True)
    w = dataclasses.replace(w, y=np.ones(w.N))
    check_log_density(torch, orc, w, precision, W.random_theta(w.dim, 50, scale=5.0, seed=44), "saturated")


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_single_fold_run(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.logistic_loo(N=400, p=5, K=1, L=4, bf16=True)
    fold = np.full(w.N, -1, np.int32)
    fold[100:140] = 0
    w = dataclasses.replace(w, fold=fold, K=1)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], batch_size=10)
    pc.warmup(100, 100)
    pc.sample(200)
    sc, dg = pc.scores(), pc.diagnostics()
    assert sc["elpd"].shape == (1,) and np.isfinite(sc["elpd_total"]) and sc["mcse_total"] > 0
    assert np.isfinite(dg["rhat_max"]) and dg["rhat_max"] < 1.2
    pc.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fold_without_test_rows_is_rejected(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_INVALID_ARG, LOGISTIC, PRECISIONS
    w = W.logistic_loo(N=100, p=3, K=10, L=2, bf16=True)
    fold = (np.arange(w.N) // 10).astype(np.int32)
    fold[fold == 4] = 5                      # fold 4 has no rows
    with pytest.raises(PCVError) as e:
        PCV(LOGISTIC, w.X, w.y, fold, 2, precision=PRECISIONS[precision])
    assert e.value.status == E_INVALID_ARG
    assert "fold 4 has no test rows" in str(e.value)
