"""Several leapfrog steps per tensor-core launch (BF16 and TF32 forms, one
CTA per 128-chain tile; lock-step HMC of Section 3.3: a tile depends on no
other tile, so its CTA can carry it from step to step): the L_f - 1
kick-drift steps of a trajectory in one launch give the same bits as one
launch per step on the same grid, and the iteration is then 4 launches
(begin, kick-drift steps, last step with the log densities, accept)
instead of L_f + 2.

* short tiles, logistic and AR(2) with log sigma sampled (its coordinate is
  finished by other epilogue threads than those that read it at the next
  step);
* config 2 itself (2000 rows: 16 BF16 or 32 TF32 chunks per tile).
The grid is fixed to one CTA per tile (tc_grid = 2) for both runs.
"""
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


def cases():
    return {
        "logistic_one_chunk": (W.logistic_loo(N=100, p=20, L=8, bf16=True), 0.02, 10),
        "ar2_one_chunk": (W.ar2_hvblock(T=130, K=5, L=8, bf16=True), 0.02, 10),
        "logistic_loo_config2": (W.logistic_loo(bf16=True), 0.02, 4),
    }


def run(w, eps, n, per_launch, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], fused_trajectory=0, tc_grid=2,
                           tc_steps_per_launch=per_launch, step_size=eps, batch_size=n // 2, acov_max_lag=4)
    truth = np.zeros(w.dim)
    tv = w.truth.get("beta", w.truth.get("phi"))
    truth[:len(tv)] = tv
    th0 = truth + 0.05 * W.random_theta(w.dim, pc.C, scale=1.0, seed=23)
    pc.set_positions(th0, step_size=eps)
    n0 = pc.kernel_launches()
    pc.sample(n)
    launches = pc.kernel_launches() - n0
    th, lp, sh = pc.positions()
    acc = pc.accept_rate()
    pc.close()
    return th, lp, sh, acc, launches


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("name", ["logistic_one_chunk", "ar2_one_chunk", "logistic_loo_config2"])
def test_steps_per_launch_same_bits(torch, name, precision):
    w, eps, n = cases()[name]
    one = run(w, eps, n, 1, precision)
    many = run(w, eps, n, 0, precision)
    for a, b in zip(one[:3], many[:3]):
        assert np.array_equal(a, b), np.abs(a - b).max()
    assert np.array_equal(np.asarray(one[3]), np.asarray(many[3]))
    assert one[4] == n * (w.leapfrog_steps + 2), one[4]
    assert many[4] == n * 4, many[4]
