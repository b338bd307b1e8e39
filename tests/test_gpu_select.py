"""GPU covariate-selection mask (Appendix B's M_j) and pairwise model
comparison (eq. sel-cv, norm-approx, mc-var): the masked model is the
sub-design model (conjugate closed form), the comparison equals the oracle's
formulas on the same fold results, and masked coefficients stay at zero on
both precisions."""
import dataclasses

import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W
from tests.test_oracle_select import closed_form_elpd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def run(w, **kw):
    from paper_2310_07002_b300.pcv import PCV
    pc = PCV.from_workload(w, **kw)
    pc.warmup(200, w.n_fold_warmup)
    pc.sample(w.n_draws)
    return pc


def test_masked_model_and_comparison(torch, orc):
    w = W.gauss_blocks()
    active = np.array([1, 1, 0, 1, 0], np.int32)
    pa = run(w)
    pb = run(dataclasses.replace(w, active=active))
    th, _, _ = pb.positions()
    assert np.all(th[:, active == 0] == 0.0)
    sb = pb.scores()
    sub = np.nonzero(active)[0]
    for k in range(w.K):
        ref = closed_form_elpd(w, k, sub)
        assert abs(sb["elpd"][k] - ref) < 4 * sb["mcse"][k], (k, sb["elpd"][k], ref)
    c = pa.compare(pb)
    sa = pa.scores()
    oc = orc.compare(sa["elpd"], sa["mcse"], sb["elpd"], sb["mcse"])
    for key in ("delta_k", "mcse_k"):
        np.testing.assert_allclose(c[key], oc[key], rtol=1e-12, atol=1e-12)
    for key in ("delta", "se", "mcse", "prob"):
        assert abs(c[key] - oc[key]) <= 1e-12 * max(1.0, abs(oc[key])), key
    full = np.arange(w.p)
    dk_ref = np.array([closed_form_elpd(w, k, full) - closed_form_elpd(w, k, sub) for k in range(w.K)])
    assert np.all(np.abs(c["delta_k"] - dk_ref) < 4 * c["mcse_k"])
    pa.close()
    pb.close()


def test_masked_coefficients_stay_zero_on_the_tensor_cores(torch):
    from paper_2310_07002_b300.pcv import PCV, BF16, PCVError, E_INVALID_ARG
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    active = np.ones(w.p, np.int32)
    active[[2, 5, 11]] = 0
    pc = PCV.from_workload(dataclasses.replace(w, active=active), precision=BF16, batch_size=10,
                          fused_trajectory=0)
    pc.warmup(60, 30)
    pc.sample(100)
    th, _, _ = pc.positions()
    assert np.all(th[:, active == 0] == 0.0) and np.all(np.abs(th[:, active == 1]).max(axis=0) > 0)
    assert pc.diagnostics()["rhat_max"] < 1.2
    pc.close()
    bad = np.ones(w.p, np.int32)
    bad[0] = 2
    with pytest.raises(PCVError) as e:
        PCV.from_workload(dataclasses.replace(w, active=bad))
    assert e.value.status == E_INVALID_ARG
