"""Checkpoint / resume: a run continued from a checkpoint in a fresh context
matches the uninterrupted run bit for bit (same Philox counters, the same
accumulator state and the same launch configurations), and a checkpoint is
refused by a context built for another problem."""
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


def state(pc):
    th, lp, sh = pc.positions()
    sc, dg = pc.scores(), pc.diagnostics()
    return [th, lp, sh, sc["elpd"], sc["mcse"], dg["rhat"], dg["split_rhat"], dg["ess_acov"],
            dg["ess_bm"], pc.accept_rate()]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_resume_continues_bit_for_bit(torch, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    kw = dict(precision=PRECISIONS[precision], batch_size=10, store_draws=200)
    a = PCV.from_workload(w, **kw)
    a.warmup(60, 30)
    a.sample(40)
    blob = a.checkpoint()
    a.sample(40)
    ref = state(a)
    ref_draws = a.draws()
    a.close()
    b = PCV.from_workload(w, **kw)
    b.restore(blob)
    b.sample(40)
    got = state(b)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)
    assert np.array_equal(b.draws(), ref_draws)
    b.close()


def test_checkpoint_refused_by_another_problem(torch):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_INVALID_ARG, E_BAD_STATE
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    a = PCV.from_workload(w, batch_size=10)
    with pytest.raises(PCVError) as e:
        a.checkpoint()                       # nothing to save before warm-up
    assert e.value.status == E_BAD_STATE
    a.warmup(20, 10)
    blob = a.checkpoint()
    a.close()
    other = PCV.from_workload(W.logistic_loo(N=517, p=20, K=31, L=4), batch_size=10)
    with pytest.raises(PCVError) as e:
        other.restore(blob)
    assert e.value.status == E_INVALID_ARG
    other.close()
    same = PCV.from_workload(w, batch_size=10)
    with pytest.raises(PCVError) as e:
        same.restore(blob[: len(blob) // 2])
    assert e.value.status == E_INVALID_ARG
    with pytest.raises(PCVError) as e:
        same.restore(b"x" * len(blob))
    assert e.value.status == E_INVALID_ARG
    same.restore(blob)
    same.sample(10)
    same.close()
