"""Failure detection without a GPU fault (host-side injections): non-finite
data and positions are refused at the boundary (E_NUMERIC); a step size far
too large makes every trajectory diverge, which the accept kernel counts
(divergences, rejections keep the chains finite); a stuck chain (one chain
started far from the others with a step too small to bring it back) is
flagged by R-hat of its fold only.  Run for the FP32 and the BF16 forms."""
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


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_non_finite_inputs_are_refused(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_NUMERIC, LOGISTIC, PRECISIONS
    w = W.logistic_loo(N=200, p=5, K=10, L=2, bf16=True)
    prec = PRECISIONS[precision]
    for bad in ("y_nan", "x_nan", "x_inf"):
        X, y = w.X.copy(), w.y.copy()
        if bad == "y_nan":
            y[17] = np.nan
        elif bad == "x_nan":
            X[3, 2] = np.nan
        else:
            X[150, 4] = np.inf
        with pytest.raises(PCVError) as e:
            PCV(LOGISTIC, X, y, w.fold, 2, precision=prec)
        assert e.value.status == E_NUMERIC, bad
    pc = PCV.from_workload(w, precision=prec)
    th = np.zeros((pc.C, w.dim))
    th[3, 1] = np.nan
    with pytest.raises(PCVError) as e:
        pc.set_positions(th, step_size=0.05)
    assert e.value.status == E_NUMERIC
    pc.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_divergent_trajectories_are_counted(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.logistic_loo(N=400, p=6, K=20, L=2, bf16=True)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], batch_size=10)
    th = np.tile(w.truth["beta"], (pc.C, 1))
    pc.set_positions(th, step_size=20.0)          # energy errors far beyond 1000
    pc.sample(50)
    dg, acc, sc = pc.diagnostics(), pc.accept_rate(), pc.scores()
    assert dg["divergences"].sum() >= 0.9 * pc.C * 50
    assert acc.max() <= 0.05
    assert np.all(np.isfinite(sc["elpd"]))        # rejected proposals leave the chains in place
    pc.close()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_stuck_chain_is_flagged_by_rhat(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.logistic_loo(N=400, p=6, K=20, L=4, bf16=True)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], batch_size=20)
    th = np.tile(w.truth["beta"], (pc.C, 1))       # every chain at one point ...
    th[4 * 7 + 2] += 3.0                           # ... but fold 7's chain 2, far from it
    pc.set_positions(th, step_size=2e-3)           # a step too small to bring it back
    pc.sample(200)
    r = pc.diagnostics()["rhat"]
    others = np.delete(r, 7)
    print("%s: rhat fold 7 %.3f, others max %.3f" % (precision, r[7], others.max()))
    assert r[7] > 2.0 and others.max() < 1.5
    pc.close()
