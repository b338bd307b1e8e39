"""GPU parity of the one-launch trajectory kernel (k_traj_small: momentum
draw, first half step and all L_f gradient steps of a chain in one warp)
against the FP64 oracle, through the C ABI, for the FP32 form and the BF16
form (a bf16 copy of the design matrix; with bf16-valued data both read the
same numbers, so the FP32 tolerances hold).

Tolerances (FP32 arithmetic, as in test_gpu_parity):
  log density after an evaluation: |d| / max(|ref|, 1) <= 1e-5;
  gradient ||d|| / ||ref|| <= 1e-5;
  one L_f-step trajectory ||d|| / ||ref|| <= 1e-4 (positions, momenta),
  log density at its end 1e-5;
  sampling follows the oracle's paths on the same Philox streams (90 % of
  chains within 1e-3 after 20 iterations, as test_sampling_follows_oracle_paths).
"""
import dataclasses

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


def rel_scalar(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


def cases():
    return {
        # 75 chains (9 full blocks of 8 warps + 3), 203 rows (6 lanes' rows + 11)
        "gauss": W.gauss_blocks(N=203, p=5, K=15, L=5, bf16=True),
        "logistic": W.logistic_loo(N=1037, p=20, K=25, L=3, bf16=True),
        "ar2": W.ar2_hvblock(T=1302, K=40, L=2, bf16=True),
        # log sigma sampled at p = 32 (the widest register tile)
        "gauss_p32": dataclasses.replace(W.gauss_blocks(N=203, p=32, K=15, L=5, bf16=True),
                                         sigma_known=-1.0, sigma_prior_sd=1.0),
        # hierarchical, leave-one-group-out: 37 groups (segments l, l + 32
        # for lanes 0 .. 4), 74 chains (9 full CTAs of 8 warps + 2)
        "hier": W.hier_logo(G=37, p=6, L=2),
    }


@pytest.mark.parametrize("wpc", [1, 8])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name", ["gauss", "logistic", "ar2", "gauss_p32", "hier"])
def test_fused_trajectory_and_evaluation(torch, orc, name, precision, wpc):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    if name == "hier" and precision == "bf16":
        pytest.skip("the hierarchical model has the FP32 form only")
    P = PRECISIONS[precision]
    w = cases()[name]
    prob = orc.problem_from_workload(w)
    eps = 0.01
    minv = np.linspace(0.5, 1.5, w.dim)
    pc = PCV.from_workload(w, precision=P, step_size=eps, inv_mass_diag=minv, fused_trajectory=wpc)
    g = np.random.Generator(np.random.Philox(61))
    # near the data-generating parameters (log sigma = 0 where sampled), so
    # that 16 steps of 0.01 stay in the stable range of the leapfrog
    truth = np.zeros(w.dim)
    tv = w.truth.get("beta", w.truth.get("phi"))
    truth[:len(tv)] = tv
    th0 = truth + 0.05 * g.standard_normal((w.n_chains, w.dim))
    r0 = g.standard_normal((w.n_chains, w.dim))
    th0 = th0.astype(np.float32).astype(np.float64)
    # the evaluation behind set_positions: log density at the start
    pc.set_positions(th0, step_size=eps, inv_mass_diag=minv)
    _, lp0, sh0 = pc.positions()
    t0 = torch.tensor(th0, dtype=torch.float32, device="cuda")
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, lp1, sh1 = pc.trajectory(t0, rr0, P)
    th1, r1 = th1.cpu().double().numpy(), r1.cpu().double().numpy()
    lp1, sh1 = lp1.cpu().numpy(), sh1.cpu().numpy()
    b0 = rr0.cpu().double().numpy()
    mv32 = minv.astype(np.float32).astype(np.float64)
    for c in range(w.n_chains):
        k = c // w.chains_per_fold
        rl, rg, rs = orc.log_density(prob, k, th0[c])
        assert rel_scalar(lp0[c], rl) <= 1e-5 and rel_scalar(sh0[c], rs) <= 1e-5, (c, lp0[c], rl)
        ref_th, ref_r, _, ref_lp, ref_sh = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps, mv32,
                                                          th0[c], b0[c], rg)
        e = (rel_vec(th1[c], ref_th), rel_vec(r1[c], ref_r), rel_scalar(lp1[c], ref_lp), rel_scalar(sh1[c], ref_sh))
        assert e[0] <= 1e-4 and e[1] <= 1e-4 and e[2] <= 1e-5 and e[3] <= 1e-5, (name, c, e)
    pc.close()


@pytest.mark.parametrize("wpc", [1, 2, 4])
@pytest.mark.parametrize("jitter", [0.0, 0.5])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_fused_sampling_follows_oracle_paths(torch, orc, precision, jitter, wpc):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.gauss_blocks(N=203, p=5, K=15, L=5, bf16=True)
    prob = orc.problem_from_workload(w)
    th0 = W.random_theta(w.dim, w.n_chains, scale=0.5, seed=41).astype(np.float32).astype(np.float64)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision], step_size=0.05, batch_size=10,
                           acov_max_lag=5, step_jitter=jitter, fused_trajectory=wpc)
    pc.set_positions(th0, step_size=0.05)
    pc.sample(20)
    th_gpu, _, sh_gpu = pc.positions()
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=0.05, b=10, M=5, jitter=jitter)
    run.set_state(th0, eps=0.05)
    run.sample(20)
    st = run.state()
    err = rel_vec(th_gpu, st["theta"])
    assert np.mean(err < 1e-3) >= 0.9, np.sort(err)[-10:]
    ok = err < 1e-3
    assert rel_scalar(sh_gpu[ok], st["shat"][ok]).max() < 1e-3
    pc.close()


def test_fused_and_separate_launches_agree(torch):
    # the same run through k_traj_small and through k_begin + L_f gradient
    # launches: different summation orders, the same chains (FP32 rounding)
    from paper_2310_07002_b300.pcv import PCV
    w = W.ar2_hvblock(T=1302, K=40, L=2)
    th0 = None
    out = {}
    for f in (0, 1, 8):
        pc = PCV.from_workload(w, step_size=0.02, batch_size=10, fused_trajectory=f)
        if th0 is None:
            th0 = np.tile(np.r_[w.truth["phi"], 0.0], (pc.C, 1)) + 0.05 * W.random_theta(w.dim, pc.C, 1.0, 5)
        pc.set_positions(th0, step_size=0.02)
        pc.sample(20)
        out[f] = pc.positions()
        pc.close()
    for f in (1, 8):
        err = rel_vec(out[0][0], out[f][0])
        assert np.mean(err < 1e-4) >= 0.9, (f, np.sort(err)[-5:])


def test_autotuner_times_the_fused_trajectory(torch, orc):
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    pc = PCV.from_workload(w, batch_size=50)
    pc.warmup(50, 50)
    info = pc.tuning_info()
    assert "trajectory for 40 chains" in info and "trajectory for 4 chains" in info, info
    pc.sample(100)
    assert np.all(np.isfinite(pc.scores()["elpd"]))
    pc.close()


@pytest.mark.parametrize("fused", [0, 1])
def test_kernel_launch_count(torch, fused):
    # the library's count of kernels issued by its iterations: one launch
    # per iteration on the fused path (trajectory, accept, accumulators),
    # k_begin + L_f gradient launches + k_accept on the separate one
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks()
    pc = PCV.from_workload(w, batch_size=10, fused_trajectory=fused)
    pc.warmup(20, 10)
    n0 = pc.kernel_launches()
    pc.sample(30)
    n = pc.kernel_launches() - n0
    pc.close()
    assert n == 30 * (1 if fused else w.leapfrog_steps + 2), n


def test_fused_hierarchical_follows_oracle_paths(torch, orc):
    # one warp per chain (z in shared memory, lanes owning whole groups):
    # 20 iterations on the same Philox streams as the oracle
    from paper_2310_07002_b300.pcv import PCV
    w = W.hier_logo(G=37, p=6, L=2)
    prob = orc.problem_from_workload(w)
    th0 = np.zeros((w.n_chains, w.dim))
    th0[:, :w.p] = w.truth["beta"]
    th0 += 0.05 * W.random_theta(w.dim, w.n_chains, scale=1.0, seed=17)
    th0 = th0.astype(np.float32).astype(np.float64)
    pc = PCV.from_workload(w, step_size=0.02, batch_size=10, acov_max_lag=5, fused_trajectory=1)
    pc.set_positions(th0, step_size=0.02)
    pc.sample(20)
    th_gpu, _, sh_gpu = pc.positions()
    pc.close()
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=0.02, b=10, M=5)
    run.set_state(th0, eps=0.02)
    run.sample(20)
    st = run.state()
    err = rel_vec(th_gpu, st["theta"])
    assert np.mean(err < 1e-3) >= 0.9, np.sort(err)[-10:]
    ok = err < 1e-3
    assert rel_scalar(sh_gpu[ok], st["shat"][ok]).max() < 1e-3


def test_fused_hierarchical_one_launch_per_iteration(torch):
    # config 3's model runs each iteration as one launch, and the fused and
    # separate paths follow the same chains
    from paper_2310_07002_b300.pcv import PCV
    w = W.hier_logo(G=37, p=6, L=2)
    th0 = np.zeros((w.n_chains, w.dim))
    th0[:, :w.p] = w.truth["beta"]
    th0 += 0.05 * W.random_theta(w.dim, w.n_chains, scale=1.0, seed=19)
    out = {}
    for f in (0, 1):
        pc = PCV.from_workload(w, step_size=0.02, batch_size=10, fused_trajectory=f)
        pc.set_positions(th0, step_size=0.02)
        n0 = pc.kernel_launches()
        pc.sample(20)
        assert pc.kernel_launches() - n0 == 20 * (1 if f else w.leapfrog_steps + 2)
        out[f] = pc.positions()[0]
        pc.close()
    err = rel_vec(out[1], out[0])
    assert np.mean(err < 1e-4) >= 0.9, np.sort(err)[-5:]
