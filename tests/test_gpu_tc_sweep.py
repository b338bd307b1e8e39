"""The BF16 tcgen05 kernel over every length of its unrolled MMA groups.

The first GEMM issues KS = ceil((p + 3) / 16) MMAs per 128-row chunk when
the centred kick-drift launches use theta's hi part only, and 2 KS when
log densities or uncentred positions need hi + lo; the second GEMM issues
two groups of four.  Each KS = 1 .. 9 (p = 13, 29, 45, 61, 77, 93, 109,
125, 128) is checked against the FP64 oracle in both forms: log density and
gradient (hi + lo: 2 KS MMAs per group) and one L_f-step trajectory on
centred positions (hi only: KS MMAs per group).

Tolerances (BF16 path, as in test_gpu_bf16): log density |d| / max(|ref|,
1) <= 1e-4, gradient ||d|| / ||ref|| <= 1e-2, trajectory 2e-2.
"""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu

PS = [13, 29, 45, 61, 77, 93, 109, 125, 128]


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


def workload(p):
    if p <= 32:
        return W.logistic_loo(N=1037, p=p, K=40, L=4, bf16=True)
    return W.logistic_large(N=1037, p=p, K=10, block=50, L=4)


@pytest.mark.parametrize("p", PS)
def test_every_mma_group_length(torch, orc, p):
    from paper_2310_07002_b300.pcv import PCV, BF16
    assert -(-(p + 3) // 16) == PS.index(p) + 1          # KS = 1 .. 9
    w = workload(p)
    prob = orc.problem_from_workload(w)
    scale = 0.3 if p <= 32 else 0.1
    # hi + lo: log densities and gradients of 300 positions (128 + 128 + 44)
    pc = PCV.from_workload(w, precision=BF16)
    n = 300
    tt = torch.tensor(W.random_theta(w.dim, n, scale=scale, seed=40 + p), dtype=torch.float32, device="cuda")
    folds = np.arange(n) % (w.K + 1)
    lp, g, _ = pc.log_density(tt, torch.tensor(folds, dtype=torch.int32, device="cuda"), BF16)
    torch.cuda.synchronize()
    lp, g = lp.cpu().numpy(), g.cpu().double().numpy()
    th = tt.cpu().double().numpy()
    for i in range(0, n, 3):
        k = int(folds[i])
        rl, rg, _ = orc.log_density(prob, -1 if k == w.K else k, th[i])
        assert rel_scalar(lp[i], rl) <= 1e-4, (p, i, lp[i], rl)
        assert rel_vec(g[i], rg) <= 1e-2, (p, i, rel_vec(g[i], rg))
    pc.close()
    # hi only: a trajectory of centred chains
    eps = 0.01 if p <= 32 else 0.004
    minv = np.ones(w.dim)
    pc = PCV.from_workload(w, precision=BF16, step_size=eps, inv_mass_diag=minv, fused_trajectory=0)
    gen = np.random.Generator(np.random.Philox(p))
    th0 = w.truth["beta"][None, :] + (0.1 if p <= 32 else 0.03) * gen.standard_normal((w.n_chains, w.dim))
    pc.set_positions(th0, step_size=eps)                   # centring reference = mean position
    r0 = gen.standard_normal((w.n_chains, w.dim))
    t0 = torch.tensor(th0, dtype=torch.float32, device="cuda")
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, _, _ = pc.trajectory(t0, rr0, BF16)
    th1, r1 = th1.cpu().double().numpy(), r1.cpu().double().numpy()
    a0, b0 = t0.cpu().double().numpy(), rr0.cpu().double().numpy()
    for c in range(0, w.n_chains, max(1, w.n_chains // 12)):
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, a0[c])
        ref_th, ref_r, _, _, _ = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps, minv, a0[c], b0[c], g0)
        assert rel_vec(th1[c], ref_th) <= 2e-2 and rel_vec(r1[c], ref_r) <= 2e-2, (p, c)
    pc.close()


PS_TF32 = [5, 13, 21, 29, 37, 45, 53, 61, 69, 77, 85, 93, 101, 109, 112]


@pytest.mark.parametrize("p", PS_TF32)
def test_every_tf32_mma_group_length(torch, orc, p):
    # the TF32 form: K steps of 8, KS = ceil((p + 3) / 8) = 1 .. 15, 64-row
    # chunks; log density and gradient of 300 positions and a trajectory of
    # centred chains, at the TF32 tolerances (log density 1e-3, gradient
    # 1e-2, trajectory 2e-2)
    from paper_2310_07002_b300.pcv import PCV, TF32
    assert -(-(p + 3) // 8) == PS_TF32.index(p) + 1
    w = workload(p)
    prob = orc.problem_from_workload(w)
    scale = 0.3 if p <= 32 else 0.1
    pc = PCV.from_workload(w, precision=TF32)
    n = 300
    tt = torch.tensor(W.random_theta(w.dim, n, scale=scale, seed=70 + p), dtype=torch.float32, device="cuda")
    folds = np.arange(n) % (w.K + 1)
    lp, g, _ = pc.log_density(tt, torch.tensor(folds, dtype=torch.int32, device="cuda"), TF32)
    torch.cuda.synchronize()
    lp, g = lp.cpu().numpy(), g.cpu().double().numpy()
    th = tt.cpu().double().numpy()
    for i in range(0, n, 3):
        k = int(folds[i])
        rl, rg, _ = orc.log_density(prob, -1 if k == w.K else k, th[i])
        assert rel_scalar(lp[i], rl) <= 1e-3, (p, i, lp[i], rl)
        assert rel_vec(g[i], rg) <= 1e-2, (p, i, rel_vec(g[i], rg))
    pc.close()
    eps = 0.01 if p <= 32 else 0.004
    minv = np.ones(w.dim)
    pc = PCV.from_workload(w, precision=TF32, step_size=eps, inv_mass_diag=minv)
    gen = np.random.Generator(np.random.Philox(p + 1000))
    th0 = w.truth["beta"][None, :] + (0.1 if p <= 32 else 0.03) * gen.standard_normal((w.n_chains, w.dim))
    pc.set_positions(th0, step_size=eps)
    r0 = gen.standard_normal((w.n_chains, w.dim))
    t0 = torch.tensor(th0, dtype=torch.float32, device="cuda")
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, _, _ = pc.trajectory(t0, rr0, TF32)
    th1, r1 = th1.cpu().double().numpy(), r1.cpu().double().numpy()
    a0, b0 = t0.cpu().double().numpy(), rr0.cpu().double().numpy()
    for c in range(0, w.n_chains, max(1, w.n_chains // 12)):
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, a0[c])
        ref_th, ref_r, _, _, _ = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps, minv, a0[c], b0[c], g0)
        assert rel_vec(th1[c], ref_th) <= 2e-2 and rel_vec(r1[c], ref_r) <= 2e-2, (p, c)
    pc.close()
