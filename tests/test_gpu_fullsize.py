"""Parity at the full size of the large logistic configuration (N = 1e5,
p = 100, K = 1000 folds x 16 chains = 16000 chains) in the launch
configurations the benchmark times: for BF16 every chain in one persistent
tcgen05 launch per leapfrog step, positions centred on a reference (hi-only
kick-drift launches); for the FP32 and TF32 forms the autotuned split-N
grid for 16000 chains (the benchmark's FP32 form), whose cross-CTA combine
differs from the small-size tests.  The FP64 oracle recomputes sampled
chains one by one over all 1e5 rows: chains at tile edges (128-chain tiles
for BF16, 64 for FP32 / TF32), in the middle and the last chain.

Tolerances:
  BF16 (as in test_gpu_bf16): log density and held-out log predictive
  |d| / max(|ref|, 1) <= 1e-4; gradient ||d|| / ||ref|| <= 1e-2; one
  L_f-step trajectory ||d|| / ||ref|| <= 2e-2 (positions and momenta).
  FP32 (as in test_gpu_parity): log density, log predictive 1e-5,
  gradient 1e-5, trajectory 1e-4.
  TF32 (as in test_gpu_tf32): 1e-3, 1e-2, 2e-2.
"""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1, 63, 64, 127, 128, 5000, 8191, 12345, 15999]

TOL = {"fp32": (1e-5, 1e-5, 1e-4), "tf32": (1e-3, 1e-2, 2e-2)}


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


@pytest.fixture(scope="module")
def large():
    return W.logistic_large()


@pytest.fixture(scope="module")
def prob(orc, large):
    return orc.problem_from_workload(large)


def rel_scalar(a, b):
    return abs(a - b) / max(abs(b), 1.0)


def rel_vec(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def positions(w, C, scale, seed):
    g = np.random.Generator(np.random.Philox(seed))
    th = np.tile(w.truth["beta"], (C, 1)) + scale * g.standard_normal((C, w.dim))
    return th


def test_fullsize_log_density_and_gradient(torch, orc, large, prob):
    from paper_2310_07002_b300.pcv import PCV, BF16
    w = large
    pc = PCV.from_workload(w, precision=BF16)
    C = pc.C
    assert C == 16000
    tt = torch.tensor(positions(w, C, 0.05, 31), dtype=torch.float32, device="cuda")
    folds = np.arange(C) // w.chains_per_fold
    lp, g, sh = pc.log_density(tt, torch.tensor(folds, dtype=torch.int32, device="cuda"), BF16)
    torch.cuda.synchronize()
    lp, g, sh = lp.cpu().numpy(), g.cpu().double().numpy(), sh.cpu().numpy()
    th = tt.cpu().double().numpy()
    for c in SAMPLE:
        rl, rg, rs = orc.log_density(prob, int(folds[c]), th[c])
        e = (rel_scalar(lp[c], rl), rel_scalar(sh[c], rs), rel_vec(g[c], rg))
        print("chain %5d: logp %.2e shat %.2e grad %.2e" % (c, *e))
        assert e[0] <= 1e-4 and e[1] <= 1e-4 and e[2] <= 1e-2
    pc.close()


def test_fullsize_centred_trajectory(torch, orc, large, prob):
    from paper_2310_07002_b300.pcv import PCV, BF16
    w = large
    eps = 0.004
    minv = np.ones(w.dim)
    pc = PCV.from_workload(w, precision=BF16, step_size=eps, inv_mass_diag=minv)
    C = pc.C
    th0 = positions(w, C, 0.05, 32)
    pc.set_positions(th0, step_size=eps)           # centring reference = mean position
    g = np.random.Generator(np.random.Philox(33))
    r0 = g.standard_normal((C, w.dim))
    t0 = torch.tensor(th0, dtype=torch.float32, device="cuda")
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, lp1, _ = pc.trajectory(t0, rr0, BF16)
    th1, r1, lp1 = th1.cpu().double().numpy(), r1.cpu().double().numpy(), lp1.cpu().numpy()
    a0, b0 = t0.cpu().double().numpy(), rr0.cpu().double().numpy()
    for c in SAMPLE[::2]:
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, a0[c])
        ref_th, ref_r, _, ref_lp, _ = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps, minv,
                                                    a0[c], b0[c], g0)
        e = (rel_vec(th1[c], ref_th), rel_vec(r1[c], ref_r), rel_scalar(lp1[c], ref_lp))
        print("chain %5d: theta %.2e r %.2e logp %.2e" % (c, *e))
        assert e[0] <= 2e-2 and e[1] <= 2e-2
        assert e[2] <= 1e-4
    pc.close()


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_fullsize_simt_and_tf32_log_density_gradient_trajectory(torch, orc, large, prob, prec):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = large
    P = PRECISIONS[prec]
    tol_lp, tol_g, tol_tr = TOL[prec]
    eps = 0.004
    minv = np.ones(w.dim)
    pc = PCV.from_workload(w, precision=P, step_size=eps, inv_mass_diag=minv)
    C = pc.C
    th0 = positions(w, C, 0.05, 34)
    pc.set_positions(th0, step_size=eps)
    pc.time_leapfrog_kernel(1)            # tunes the split-N grid for 16000 chains, as the benchmark does
    assert "16000 chains" in pc.tuning_info()
    tt = torch.tensor(th0, dtype=torch.float32, device="cuda")
    folds = np.arange(C) // w.chains_per_fold
    lp, g, sh = pc.log_density(tt, torch.tensor(folds, dtype=torch.int32, device="cuda"), P)
    torch.cuda.synchronize()
    lp, g, sh = lp.cpu().numpy(), g.cpu().double().numpy(), sh.cpu().numpy()
    th = tt.cpu().double().numpy()
    for c in SAMPLE:
        rl, rg, rs = orc.log_density(prob, int(folds[c]), th[c])
        e = (rel_scalar(lp[c], rl), rel_scalar(sh[c], rs), rel_vec(g[c], rg))
        print("%s chain %5d: logp %.2e shat %.2e grad %.2e" % (prec, c, *e))
        assert e[0] <= tol_lp and e[1] <= tol_lp and e[2] <= tol_g
    g = np.random.Generator(np.random.Philox(35))
    r0 = g.standard_normal((C, w.dim))
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, lp1, _ = pc.trajectory(tt, rr0, P)
    th1, r1, lp1 = th1.cpu().double().numpy(), r1.cpu().double().numpy(), lp1.cpu().numpy()
    b0 = rr0.cpu().double().numpy()
    for c in SAMPLE[::3]:
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, th[c])
        ref_th, ref_r, _, ref_lp, _ = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps, minv,
                                                    th[c], b0[c], g0)
        e = (rel_vec(th1[c], ref_th), rel_vec(r1[c], ref_r), rel_scalar(lp1[c], ref_lp))
        print("%s chain %5d: theta %.2e r %.2e logp %.2e" % (prec, c, *e))
        assert e[0] <= tol_tr and e[1] <= tol_tr and e[2] <= tol_lp
    pc.close()
