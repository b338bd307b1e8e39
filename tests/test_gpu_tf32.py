"""GPU parity of the TF32 rung (tcgen05 kind::tf32 tensor cores: theta,
X and the residual rounded to TF32, FP32 accumulation) against the FP64
oracle, through the C ABI.  TF32 keeps 10 mantissa bits, so the tolerances
are those of a reduced-precision form (stated and asserted here):
  log density, held-out log predictive: |d| / max(|ref|, 1) <= 1e-3
  gradient: ||d||_2 / ||ref||_2 <= 1e-2
  one L_f-step trajectory: ||d||_2 / ||ref||_2 <= 2e-2
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


def workloads():
    return {
        # 1037 rows: 16 chunks of 64 + 13; 130 positions: 2 chain tiles + 2
        "logistic_p20": W.logistic_loo(N=1037, p=20, K=40, L=4),
        "logistic_p100": W.logistic_large(N=1037, p=100, K=10, block=50, L=4),
        "gauss": W.gauss_blocks(N=203, p=5, K=15, L=5),
        "gauss_p40": dataclasses.replace(W.gauss_blocks(N=203, p=40, K=15, L=5),
                                         sigma_known=-1.0, sigma_prior_sd=1.0),
    }


@pytest.mark.parametrize("name", ["logistic_p20", "logistic_p100", "gauss", "gauss_p40"])
def test_tf32_log_density_and_gradient(torch, orc, name):
    from paper_2310_07002_b300.pcv import PCV, TF32
    w = workloads()[name]
    pc = PCV.from_workload(w, precision=TF32)
    prob = orc.problem_from_workload(w)
    n = 130
    scale = 0.3 if w.p <= 32 else 0.1
    tt = torch.tensor(W.random_theta(w.dim, n, scale=scale, seed=29), dtype=torch.float32, device="cuda")
    folds = np.arange(n) % (w.K + 1)
    fo = torch.tensor(folds, dtype=torch.int32, device="cuda")
    lp, g, sh = pc.log_density(tt, fo, TF32)
    torch.cuda.synchronize()
    lp, g, sh = lp.cpu().numpy(), g.cpu().double().numpy(), sh.cpu().numpy()
    th = tt.cpu().double().numpy()
    ref = [orc.log_density(prob, -1 if k == w.K else int(k), th[i]) for i, k in enumerate(folds)]
    lp_ref = np.array([r[0] for r in ref]); g_ref = np.stack([r[1] for r in ref])
    sh_ref = np.array([r[2] for r in ref])
    print(name, rel_scalar(lp, lp_ref).max(), rel_vec(g, g_ref).max(), rel_scalar(sh, sh_ref).max())
    assert rel_scalar(lp, lp_ref).max() <= 1e-3
    assert rel_scalar(sh, sh_ref).max() <= 1e-3
    assert rel_vec(g, g_ref).max() <= 1e-2
    pc.close()


# grid 2: one CTA per tile, so the kick-drift steps of the trajectory run in
# one launch (theta reaches TMEM after each step's finish)
@pytest.mark.parametrize("grid", [0, 2])
@pytest.mark.parametrize("name", ["logistic_p100", "gauss_p40"])
def test_tf32_trajectory(torch, orc, name, grid):
    from paper_2310_07002_b300.pcv import PCV, TF32
    w = workloads()[name]
    eps = 0.004 if name == "logistic_p100" else 0.002
    minv = np.linspace(0.5, 1.5, w.dim)
    pc = PCV.from_workload(w, precision=TF32, step_size=eps, inv_mass_diag=minv, tc_grid=grid)
    prob = orc.problem_from_workload(w)
    g = np.random.Generator(np.random.Philox(7))
    t0 = torch.tensor(0.05 * g.standard_normal((w.n_chains, w.dim)), dtype=torch.float32, device="cuda")
    r0 = torch.tensor(g.standard_normal((w.n_chains, w.dim)), dtype=torch.float32, device="cuda")
    th1, r1, lp1, _ = pc.trajectory(t0, r0, TF32)
    th1, r1 = th1.cpu().double().numpy(), r1.cpu().double().numpy()
    th0 = t0.cpu().double().numpy(); rr0 = r0.cpu().double().numpy()
    ref_th = np.empty_like(th1); ref_r = np.empty_like(r1)
    for c in range(w.n_chains):
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, th0[c])
        ref_th[c], ref_r[c], _, _, _ = orc.trajectory(prob, k, np.float32(eps), w.leapfrog_steps,
                                                      minv.astype(np.float32).astype(np.float64),
                                                      th0[c], rr0[c], g0)
    assert rel_vec(th1, ref_th).max() <= 2e-2
    assert rel_vec(r1, ref_r).max() <= 2e-2
    pc.close()


def test_tf32_and_fp32_runs_agree(torch):
    from paper_2310_07002_b300.pcv import PCV, TF32, FP32_SIMT
    w = W.logistic_loo(N=600, p=12, K=24, L=8, bf16=True)
    out = {}
    for prec in (FP32_SIMT, TF32):
        pc = PCV.from_workload(w, precision=prec)
        pc.warmup(300, 300)
        pc.sample(2000)
        out[prec] = (pc.scores(), pc.diagnostics())
        pc.close()
    (s32, d32), (st, dt) = out[FP32_SIMT], out[TF32]

    def mcse(s, d):
        return s["mcse"] * np.sqrt(np.maximum(1.0, d["ess_bm"] / d["ess_acov"]))
    z = np.abs(s32["elpd"] - st["elpd"]) / np.sqrt(mcse(s32, d32) ** 2 + mcse(st, dt) ** 2)
    zt = abs(s32["elpd_total"] - st["elpd_total"]) / np.hypot(s32["mcse_total"], st["mcse_total"])
    assert zt < 4.0 and z.max() < 5.0 and z.mean() < 1.3
    assert dt["rhat_max"] < 1.05


def test_tf32_rejects_the_hierarchical_model(torch):
    from paper_2310_07002_b300.pcv import PCV, TF32, PCVError, E_UNSUPPORTED
    with pytest.raises(PCVError) as e:
        PCV.from_workload(W.hier_logo(G=10, p=3, L=2), precision=TF32)
    assert e.value.status == E_UNSUPPORTED
