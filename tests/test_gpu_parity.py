"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
identical seeded inputs.

Tolerances (stated for FP32 kernels):
  log density, held-out log predictive: |d| / max(|ref|, 1) <= 1e-5
  gradient: ||d||_2 / ||ref||_2 <= 1e-5 per position
  one L_f-step trajectory: ||d||_2 / ||ref||_2 <= 1e-4 (positions and momenta)
  normals: |d| <= 2e-6 (FP32 Box-Muller vs FP64)
  accumulators / estimators (FP64 on both sides): rtol 1e-9
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


def small_workloads():
    return {
        # ragged: 75 chains = 2 full tiles of 32 + 11; N not a multiple of anything
        "gauss": W.gauss_blocks(N=203, p=5, K=15, L=5),
        "logistic": W.logistic_loo(N=1037, p=20, K=25, L=3),
        "ar2": W.ar2_hvblock(T=1302, K=40, L=2),
        "hier": W.hier_logo(G=23, p=10, L=3, mean_extra=12.0),
        # p > 32 takes the shared-memory-tiled FP32 kernel (64-chain tiles):
        # 78 chains = 64 + 14, 1037 rows = 32 chunks of 32 + 13
        "logistic_p100": W.logistic_loo(N=1037, p=100, K=25, L=3),
        # Gaussian with sampled log sigma at p = 40 (gradient slot after beta)
        "gauss_p40": dataclasses.replace(W.gauss_blocks(N=203, p=40, K=15, L=5),
                                         sigma_known=-1.0, sigma_prior_sd=1.0),
    }


def make_pcv(w, **kw):
    from paper_2310_07002_b300.pcv import PCV
    return PCV.from_workload(w, **kw)


def rel_scalar(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


@pytest.mark.parametrize("name", ["gauss", "logistic", "ar2", "hier", "logistic_p100", "gauss_p40"])
def test_log_density_and_gradient(torch, orc, name):
    w = small_workloads()[name]
    pc = make_pcv(w)
    prob = orc.problem_from_workload(w)
    n = 3 * (w.K + 1) + 1
    th = W.random_theta(w.dim, n, scale=0.3, seed=17)
    folds = np.arange(n) % (w.K + 1)               # includes K = full data
    lp_ref = np.empty(n); sh_ref = np.empty(n); g_ref = np.empty((n, w.dim))
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    # the oracle evaluates at the FP32-rounded positions the GPU sees
    th32 = tt.cpu().double().numpy()
    for i in range(n):
        k = int(folds[i])
        lp_ref[i], g_ref[i], sh_ref[i] = orc.log_density(prob, -1 if k == w.K else k, th32[i])
    fo = torch.tensor(folds, dtype=torch.int32, device="cuda")
    lp, g, sh = pc.log_density(tt, fo)
    torch.cuda.synchronize()
    lp, g, sh = lp.cpu().numpy(), g.cpu().double().numpy(), sh.cpu().numpy()
    assert rel_scalar(lp, lp_ref).max() <= 1e-5
    assert rel_scalar(sh, sh_ref).max() <= 1e-5
    assert rel_vec(g, g_ref).max() <= 1e-5
    pc.close()


def test_normals_match_oracle(torch, orc):
    w = small_workloads()["gauss"]
    pc = make_pcv(w)
    for it, st in [(0, 0), (5, 0), (3, 16)]:
        z = pc.draw_normals(it, st).cpu().double().numpy()
        ref = np.stack([orc.normals(w.seed, c, it, st, w.dim) for c in range(w.n_chains)])
        assert np.abs(z - ref).max() <= 2e-6
    pc.close()


@pytest.mark.parametrize("name", ["gauss", "logistic", "ar2", "hier", "logistic_p100", "gauss_p40"])
def test_single_trajectory(torch, orc, name):
    w = small_workloads()[name]
    eps = {"gauss": 0.01, "logistic": 0.01, "ar2": 0.005, "hier": 0.01, "logistic_p100": 0.004,
           "gauss_p40": 0.002}[name]
    minv = np.linspace(0.5, 1.5, w.dim)
    pc = make_pcv(w, step_size=eps, inv_mass_diag=minv)
    prob = orc.problem_from_workload(w)
    g = np.random.Generator(np.random.Philox(5))
    th0 = 0.2 * g.standard_normal((w.n_chains, w.dim))
    r0 = g.standard_normal((w.n_chains, w.dim))
    t0 = torch.tensor(th0, dtype=torch.float32, device="cuda")
    rr0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    th1, r1, lp1, sh1 = pc.trajectory(t0, rr0)
    th1, r1, lp1 = th1.cpu().double().numpy(), r1.cpu().double().numpy(), lp1.cpu().numpy()
    th0_32 = t0.cpu().double().numpy()
    r0_32 = rr0.cpu().double().numpy()
    ref_th = np.empty_like(th1); ref_r = np.empty_like(r1); ref_lp = np.empty(w.n_chains)
    for c in range(w.n_chains):
        k = c // w.chains_per_fold
        _, g0, _ = orc.log_density(prob, k, th0_32[c])
        ref_th[c], ref_r[c], _, ref_lp[c], _ = orc.trajectory(
            prob, k, np.float32(eps), w.leapfrog_steps, minv.astype(np.float32).astype(np.float64),
            th0_32[c], r0_32[c], g0)
    assert rel_vec(th1, ref_th).max() <= 1e-4
    assert rel_vec(r1, ref_r).max() <= 1e-4
    assert rel_scalar(lp1, ref_lp).max() <= 1e-4
    pc.close()


def test_accumulators_match_oracle(torch, orc):
    w = small_workloads()["gauss"]
    L, b, M = w.chains_per_fold, 25, 20
    pc = make_pcv(w, batch_size=b, acov_max_lag=M)
    pc.set_positions(np.zeros((w.n_chains, w.dim)), step_size=0.01)
    s = W.random_shat_series(w.n_chains, 300, rho=0.6, loc=-40.0, scale=2.0, seed=31)
    pc.accumulate(torch.tensor(s[:, :150], device="cuda"))
    pc.accumulate(torch.tensor(s[:, 150:], device="cuda"))      # two calls = progressive
    sc = pc.scores()
    dg = pc.diagnostics()
    fo, to = orc.accumulate_series(s, L, b, M)
    np.testing.assert_allclose(sc["elpd"], fo["elpd"], rtol=1e-10)
    np.testing.assert_allclose(sc["mcse"], fo["mcse"], rtol=1e-9)
    np.testing.assert_allclose(dg["rhat"], fo["rhat"], rtol=1e-10)
    np.testing.assert_allclose(dg["split_rhat"], fo["split_rhat"], rtol=1e-10)
    np.testing.assert_allclose(dg["ess_bm"], fo["ess_bm"], rtol=1e-9)
    np.testing.assert_allclose(dg["ess_acov"], fo["ess_acov"], rtol=1e-9)
    assert abs(sc["elpd_total"] - to["elpd"]) < 1e-9
    assert abs(sc["mcse_total"] - to["mcse"]) < 1e-12
    assert abs(sc["se_epistemic"] - to["se_epistemic"]) < 1e-9
    assert abs(dg["rhat_max"] - to["rhat_max"]) < 1e-12
    assert abs(dg["ess_total"] / to["ess_total"] - 1) < 1e-9
    pc.close()


def test_autograd_function_vs_finite_differences(torch, orc):
    from paper_2310_07002_b300.pcv import masked_log_density
    w = small_workloads()["logistic"]
    pc = make_pcv(w)
    th = torch.tensor(W.random_theta(w.dim, 4, scale=0.2, seed=3), dtype=torch.float32,
                      device="cuda", requires_grad=True)
    fo = torch.tensor([0, 5, 24, w.K], dtype=torch.int32, device="cuda")
    lp = masked_log_density(th, pc, fo)
    weights = torch.tensor([1.0, -0.5, 2.0, 0.25], dtype=torch.float64, device="cuda")
    (lp * weights).sum().backward()
    gk = th.grad.cpu().double().numpy()
    # central differences of the kernel's own log density, step 1e-2 per coordinate
    base = th.detach().cpu().double().numpy()
    h = 1e-2
    fd = np.zeros_like(base)
    for j in range(w.dim):
        tp = base.copy(); tp[:, j] += h
        tm = base.copy(); tm[:, j] -= h
        lpp = pc.log_density(torch.tensor(tp, dtype=torch.float32, device="cuda"), fo)[0].cpu().numpy()
        lpm = pc.log_density(torch.tensor(tm, dtype=torch.float32, device="cuda"), fo)[0].cpu().numpy()
        fd[:, j] = (lpp - lpm) / (2 * h) * weights.cpu().numpy()
    assert rel_vec(gk, fd).max() < 2e-3
    # and against the oracle's analytic gradient
    prob = orc.problem_from_workload(w)
    for i, k in enumerate([0, 5, 24, -1]):
        _, g, _ = orc.log_density(prob, k, base[i])
        assert rel_vec(gk[i] / weights[i].item(), g) < 1e-5
    pc.close()


def test_sampling_follows_oracle_paths(torch, orc):
    # Same start, same Philox streams: FP32 GPU chains track the FP64 oracle's
    # chains transition by transition until an accept decision near its
    # threshold flips; most chains must stay on the oracle's path.
    w = W.gauss_blocks(N=203, p=5, K=15, L=5)
    prob = orc.problem_from_workload(w)
    th0 = W.random_theta(w.dim, w.n_chains, scale=0.5, seed=41)
    th0 = th0.astype(np.float32).astype(np.float64)
    pc = make_pcv(w, step_size=0.05, batch_size=10, acov_max_lag=5)
    pc.set_positions(th0, step_size=0.05)
    pc.sample(20)
    th_gpu, lp_gpu, sh_gpu = pc.positions()
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=0.05, b=10, M=5)
    run.set_state(th0, eps=0.05)
    run.sample(20)
    st = run.state()
    err = rel_vec(th_gpu, st["theta"])
    assert np.mean(err < 1e-3) >= 0.9, np.sort(err)[-10:]
    ok = err < 1e-3
    assert rel_scalar(sh_gpu[ok], st["shat"][ok]).max() < 1e-3
    pc.close()


def test_conjugate_run_matches_closed_form(torch, orc):
    from tests.test_oracle_conjugate import closed_form
    w = W.gauss_blocks()
    pc = make_pcv(w)
    pc.warmup(200, w.n_fold_warmup)
    pc.sample(w.n_draws)
    sc = pc.scores()
    dg = pc.diagnostics()
    for k in range(w.K):
        _, _, elpd = closed_form(w, k)
        assert abs(sc["elpd"][k] - elpd) < 4 * sc["mcse"][k], (k, sc["elpd"][k], elpd, sc["mcse"][k])
    assert dg["rhat_max"] < 1.05
    assert pc.accept_rate().min() > 0.5
    assert dg["divergences"].sum() == 0
    # statistical agreement with a whole oracle run (different draws: combined MCSE)
    prob = orc.problem_from_workload(w)
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=w.step_size, b=50)
    run.fulldata(200, 250)
    run.fold_warmup(w.n_fold_warmup)
    run.sample(w.n_draws)
    fo, _ = run.results()
    comb = np.sqrt(sc["mcse"] ** 2 + fo["mcse"] ** 2)
    assert np.all(np.abs(sc["elpd"] - fo["elpd"]) < 4 * comb)
    pc.close()


def test_adapted_warmup_is_sane(torch, orc):
    w = W.logistic_loo(N=400, p=6, K=20, L=4)
    pc = make_pcv(w, step_size=-1.0)
    pc.warmup(300, 200)
    eps, minv = pc.adaptation()
    # the adapted step size is capped so that L_f steps span pi/2
    assert 1e-3 < eps <= np.pi / 2 / w.leapfrog_steps * (1 + 1e-6) and np.all(minv > 0)
    pc.sample(500)
    assert 0.5 < pc.accept_rate().mean() <= 1.0
    assert pc.diagnostics()["rhat_max"] < 1.05
    pc.close()


def test_jittered_sampling_follows_oracle_paths(torch, orc):
    # one step size per iteration, eps (1 + j (2u - 1)) with u from Philox
    # stream 3, shared by all chains: the GPU and the oracle draw the same u
    w = W.gauss_blocks(N=203, p=5, K=15, L=5)
    prob = orc.problem_from_workload(w)
    th0 = W.random_theta(w.dim, w.n_chains, scale=0.5, seed=43)
    th0 = th0.astype(np.float32).astype(np.float64)
    pc = make_pcv(w, step_size=0.05, batch_size=10, acov_max_lag=5, step_jitter=0.5)
    pc.set_positions(th0, step_size=0.05)
    pc.sample(20)
    th_gpu, _, sh_gpu = pc.positions()
    run = orc.OraclePCV(prob, w.chains_per_fold, w.seed, w.leapfrog_steps, eps=0.05, b=10, M=5,
                        jitter=0.5)
    run.set_state(th0, eps=0.05)
    run.sample(20)
    st = run.state()
    err = rel_vec(th_gpu, st["theta"])
    assert np.mean(err < 1e-3) >= 0.9, np.sort(err)[-10:]
    # without the jitter on the GPU side the paths part at once
    pc2 = make_pcv(w, step_size=0.05, batch_size=10, acov_max_lag=5, step_jitter=0.0)
    pc2.set_positions(th0, step_size=0.05)
    pc2.sample(20)
    assert np.mean(rel_vec(pc2.positions()[0], st["theta"]) < 1e-3) < 0.5
    pc.close()
    pc2.close()


def test_error_codes(torch):
    from paper_2310_07002_b300.pcv import PCV, PCVError, E_BAD_STATE, E_INVALID_ARG
    w = W.gauss_blocks(N=60, p=3, K=3, L=2)
    pc = make_pcv(w)
    with pytest.raises(PCVError) as e:
        pc.sample(50)
    assert e.value.status == E_BAD_STATE
    with pytest.raises(PCVError) as e:
        pc.scores()
    assert e.value.status == E_BAD_STATE
    pc.set_positions(np.zeros((w.n_chains, w.dim)), step_size=0.05)
    with pytest.raises(PCVError) as e:
        pc.sample(49)                      # not a multiple of the batch size
    assert e.value.status == E_INVALID_ARG
    pc.close()
    # a fold whose test block covers every row has no training rows
    f = np.zeros(w.N, np.int32)
    with pytest.raises(PCVError) as e:
        PCV(0, w.X, w.y, f, 2, beta_prior_sd=10.0, sigma_known=1.0)
    assert e.value.status == E_INVALID_ARG
    # h(v)-block folds must be contiguous
    f = np.full(w.N, -1, np.int32)
    f[[3, 9]] = 0
    with pytest.raises(PCVError) as e:
        PCV(3, w.X, w.y, f, 2, hv_buffer=2)
    assert e.value.status == E_INVALID_ARG


@pytest.mark.parametrize("fused", [0, 1])
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_graph_replay_equals_plain_launches(torch, precision, fused):
    # The iteration replayed from a captured CUDA graph (counters in device
    # memory) must produce bit-identical states and estimators to the same
    # launches issued one by one.
    from paper_2310_07002_b300.pcv import PRECISIONS
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    out = []
    for graphs in (True, False):
        # a fixed launch configuration: the autotuner's choice of split count
        # could differ between the two contexts and change rounding
        pc = make_pcv(w, precision=PRECISIONS[precision], use_graphs=graphs, batch_size=10,
                      autotune=False, fused_trajectory=fused)
        pc.warmup(40, 20)
        pc.sample(60)
        th, lp, sh = pc.positions()
        sc = pc.scores()
        dg = pc.diagnostics()
        out.append((th, lp, sh, sc["elpd"], dg["rhat"], dg["ess_acov"]))
        su = pc.setup_ms()
        assert su["autotune_ms"] == 0.0 and (su["graph_capture_ms"] > 0.0) == graphs, su
        pc.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_autotuner_records_its_choice_and_results_hold(torch, orc, precision):
    from paper_2310_07002_b300.pcv import PRECISIONS
    w = W.logistic_loo(N=517, p=20, K=30, L=4)
    pc = make_pcv(w, precision=PRECISIONS[precision], batch_size=10)
    pc.warmup(40, 20)
    info = pc.tuning_info()
    assert "->" in info and "chains" in info, info
    # its wall clock and the graph captures' are kept apart from the run's
    su = pc.setup_ms()
    assert su["autotune_ms"] > 0.0 and su["graph_capture_ms"] > 0.0, su
    # the tuned launch still computes the oracle's gradient
    prob = orc.problem_from_workload(w)
    th = W.random_theta(w.dim, pc.C, scale=0.3, seed=3)
    tt = torch.tensor(th, dtype=torch.float32, device="cuda")
    fo = torch.tensor(np.arange(pc.C) // w.chains_per_fold, dtype=torch.int32, device="cuda")
    lp, g, _ = pc.log_density(tt, fo, precision=PRECISIONS[precision])
    th32 = tt.cpu().double().numpy()
    ref = np.stack([orc.log_density(prob, int(k), th32[i])[1] for i, k in enumerate(fo.cpu().numpy())])
    tol = 1e-5 if precision == "fp32" else 1e-2
    assert rel_vec(g.cpu().double().numpy(), ref).max() <= tol
    pc.close()


def test_fold_shards_draw_the_streams_of_their_global_folds(torch):
    # a context that owns folds k0..K-1 of a problem (rows of other folds
    # train only) with first_fold = k0 follows the single-context paths of
    # those folds; with first_fold = 0 it draws other random numbers
    from paper_2310_07002_b300 import shard
    from paper_2310_07002_b300.pcv import PCV
    w = W.gauss_blocks(N=203, p=5, K=15, L=5)
    L, k0 = w.chains_per_fold, 8
    th0 = W.random_theta(w.dim, w.n_chains, scale=0.5, seed=47).astype(np.float32).astype(np.float64)
    full = make_pcv(w, step_size=0.05, batch_size=10, autotune=False)
    full.set_positions(th0, step_size=0.05)
    full.sample(10)
    ref = full.positions()[0][k0 * L:]
    full.close()
    sub = dataclasses.replace(w, fold=shard.shard_folds(w.fold, k0, w.K), K=w.K - k0)
    out = {}
    for ff in (k0, 0):
        pc = make_pcv(sub, step_size=0.05, batch_size=10, autotune=False, first_fold=ff)
        pc.set_positions(th0[k0 * L:], step_size=0.05)
        pc.sample(10)
        out[ff] = rel_vec(pc.positions()[0], ref)
        pc.close()
    assert np.mean(out[k0] < 1e-4) >= 0.9, np.sort(out[k0])[-5:]
    assert np.mean(out[0] < 1e-4) < 0.2
