#!/usr/bin/env python3
"""PCV throughput benchmark: leapfrog gradient evaluations per second over
all fold-chains (one step = one lock-step HMC iteration of every chain:
momentum draw, L_f fused gradient+update launches, FP64 accept and the
online accumulators).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision fp32|bf16|tf32] [--no-fp32-form]

Default: the large random-block logistic workload (N=1e5, p=100, K=1000
folds x 16 chains) in BF16 on the tensor cores, with the plain FP32 form
timed beside it on the same GPU (`fp32_form`).

Multi-GPU (torchrun, one rank per GPU): each rank runs its own copy of the
workload with its own sampler seed (folds are independent posteriors, so the
path shards with no data-path collective; weak scaling).  Rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2310_07002_b300 import workloads as W  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 CUDA-core peak: 148 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.032 GHz
FP32_SIMT_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12

WORKLOADS = {
    "logistic_loo": lambda: W.logistic_loo(),        # N=2000, p=20, K=2000, L=8
    "logistic_large": lambda: W.logistic_large(),    # N=1e5, p=100, K=1000, L=16
    # a quarter-size case of the same kernel for multi-pass profiler captures
    "logistic_large_q": lambda: W.logistic_large(N=25_000, K=250),
    "gauss_blocks": lambda: W.gauss_blocks(),
    "hier_logo": lambda: W.hier_logo(),
    "ar2_hvblock": lambda: W.ar2_hvblock(),
}


# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), with the SHA-256 of
# the kernel's source files at capture time: a figure whose sources have
# changed since is not reported (traffic: null).
TC_SOURCES = ("k_grad_tc.cu", "tc_ptx.cuh")
TRAFFIC = {
    # kick-drift launch of the tcgen05 kernel (k_grad_tc<7, false, false>)
    ("logistic_large", "bf16"): (42.97e6, TC_SOURCES, "6ae17755755e2bf7"),
    # kick-drift launch of the TF32 tcgen05 kernel (k_grad_tc<13, false, false, true>)
    ("logistic_large", "tf32"): (131.23e6, TC_SOURCES, "6ae17755755e2bf7"),
    # FP32 shared-memory-tiled kernel (k_grad_bigp<MV_LOGISTIC>)
    ("logistic_large", "fp32"): (48.93e6, ("k_grad_simt.cu",), None),
}


def sources_sha(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2310_07002_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_of(workload: str, precision: str):
    ent = TRAFFIC.get((workload, precision))
    if ent is None or ent[0] is None or ent[2] is None:
        return None
    return ent[0] if sources_sha(ent[1]).startswith(ent[2]) else None


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def flops_per_grad_eval(w) -> float:
    """Algorithmic flops of one masked log-density gradient for one chain:
    2 N p for x'beta over all N rows and 2 N p for X'r (Appendix B masking
    evaluates every row)."""
    return 4.0 * w.N * w.p


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(w, seconds: float, n_chains_target: int, threads: int):
    """Oracle (as it stands) on a bounded sample of the workload: the first
    folds' chains over all N rows, started at the data-generating parameters.
    Returns (grad-evals/s, description, cores)."""
    import oracle
    L = w.chains_per_fold
    n_folds = max(1, n_chains_target // L)
    sub_fold = np.where((w.fold >= 0) & (w.fold < n_folds), w.fold, -1).astype(np.int32)
    prob = oracle.oracle._ProblemHolder(w.kind, w.X, w.y, sub_fold, n_folds, w.hv_buffer, w.group,
                                        w.n_groups, w.beta_prior_sd, w.sigma_known,
                                        w.sigma_prior_sd, w.tau_prior_sd)
    d = prob.dim
    th = np.zeros((n_folds * L, d))
    truth = w.truth.get("beta", w.truth.get("phi"))
    if truth is not None:
        th[:, :len(truth)] = truth
    run = oracle.OraclePCV(prob, L, w.seed, w.leapfrog_steps, eps=1e-3, b=1,
                           max_batches=1 << 16, n_threads=threads)
    run.set_state(th, eps=1e-3)
    iters = 0
    t0 = time.perf_counter()
    while True:
        run.sample(1)
        iters += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    evals = n_folds * L * w.leapfrog_steps * iters
    desc = ("%d folds x %d chains x %d iterations (%d leapfrog steps each) over all %d rows"
            % (n_folds, L, iters, w.leapfrog_steps, w.N))
    return evals / el, desc, threads


def bench_config(w, args):
    """The workload description both arms print (the reference arm times the
    same workload, so its `config` is this arm's)."""
    return {"workload": w.name, "N": w.N, "p": w.p, "K": w.K, "L": w.chains_per_fold,
            "chains": w.K * w.chains_per_fold, "leapfrog_steps": w.leapfrog_steps,
            "precision": args.precision,
            "l2": "flushed (256 MB write) before every timed step",
            "parallelism": "replica per GPU (independent fold-chains)"}


def run_reference(args, w):
    """Reference arm: the FP64 oracle on the host cores, bounded samples."""
    threads = os.cpu_count() or 1
    per_step = max(0.5, min(5.0, 150.0 / max(1, args.steps + args.warmup)))
    target = 64 if w.N * w.p < 1e6 else 16
    oracle_rate(w, 0.2, target, threads)               # warm-up (page-in, threads)
    rates = []
    desc = ""
    for _ in range(args.steps):
        r, desc, _ = oracle_rate(w, per_step, target, threads)
        rates.append(r)
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": "leapfrog grad-evals/s over all fold-chains",
        "value": value, "unit": "grad-evals/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, args),
        "cpu_baseline": {"value": value, "unit": "grad-evals/s", "cores": threads,
                         "kind": "oracle", "sample": "each step: " + desc},
        "e2e": {"value": value, "unit": "grad-evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(P, w, prec, K, Wu, seed, barrier, flush, nvtx=True, fused=-1, tc_grid=0):
    """Create a context for workload w at precision prec, run Wu untimed
    warm-up iterations, then time K sampling iterations (one step each) with
    CUDA events on the library's launch stream, L2 flushed before each step.
    The fused leapfrog launch is also timed on its own (20 back-to-back
    launches on the proposal buffers; the chains' state is not touched):
    before the timed steps after a second at rest, the state a burst peak is
    measured in, and right after them, where the long run has brought the
    power cap in.  Returns (total_ms, chains, kernel_ms rested, kernel_ms
    after the steps, launches)."""
    import time
    import torch
    common = dict(seed=seed, batch_size=1, max_batches=K + 64, acov_max_lag=64,
                  precision=prec, init_scale=0.1, fused_trajectory=fused, tc_grid=tc_grid)
    pc = P.PCV.from_workload(w, **common)
    pc.warmup(100, Wu)                                   # untimed warm-up iterations
    stream = pc.stream
    torch.cuda.synchronize()
    time.sleep(1.0)
    k_ms = pc.time_leapfrog_kernel(20)
    barrier()
    n0 = pc.kernel_launches()
    step_ms = []
    if nvtx:
        torch.cuda.nvtx.range_push("pcv_timed")         # lets a profiler select these launches
    for _ in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        pc.sample(1)                                     # CUDA events on the launch stream
        step_ms.append(pc.last_sample_ms())
    if nvtx:
        torch.cuda.nvtx.range_pop()
    barrier()
    launches = pc.kernel_launches() - n0                # our kernels in the timed region
    k_ms_hot = pc.time_leapfrog_kernel(20)
    C = pc.C
    pc.close()
    return float(np.sum(step_ms)), C, k_ms, k_ms_hot, launches


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="logistic_large", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16", choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-form", action="store_true",
                    help="skip timing the plain FP32 form beside a BF16/TF32 run")
    ap.add_argument("--tc-grid", type=int, default=0, choices=[0, 1, 2],
                    help="tensor-core grid: 0 autotuned, 1 one CTA per SM (tiles split), 2 one CTA per tile "
                         "(fixes the choice for profiler runs)")
    ap.add_argument("--fused-trajectory", type=int, default=-1, choices=[-1, 0, 1, 2, 4, 8],
                    help="whole trajectories in one launch: -1 autotuned (default), 0 never, w > 0 always "
                         "with w warps per chain where the problem allows (fixes the choice for profiler runs)")
    ap.add_argument("--profile-launches", action="store_true",
                    help="for profiler captures: create the context, set positions and "
                         "autotune, then inside NVTX range pcv_prof one gradient launch "
                         "with log densities and three kick-drift gradient launches; "
                         "prints no JSON line")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOADS[args.workload]()

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, w)
        return

    import torch
    from paper_2310_07002_b300.build import build
    from paper_2310_07002_b300 import pcv as P
    build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    prec = P.PRECISIONS[args.precision]
    if args.profile_launches:
        pc = P.PCV.from_workload(w, precision=prec, tc_grid=args.tc_grid)
        theta0 = np.zeros((pc.C, w.dim))
        truth = w.truth.get("beta", w.truth.get("phi"))
        if truth is not None:
            theta0[:, :len(truth)] = truth
        pc.set_positions(theta0, step_size=1e-3)
        pc.time_leapfrog_kernel(1)          # autotuner (launch configuration of the timed runs)
        torch.cuda.synchronize()
        # the launches to profile, inside NVTX range pcv_prof: one gradient
        # evaluation with log densities (set_positions), then kick-drift
        # launches in the tuned configuration
        torch.cuda.nvtx.range_push("pcv_prof")
        pc.set_positions(theta0, step_size=1e-3)
        ms = pc.time_leapfrog_kernel(2)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        pc.close()
        print("profile launches done: %.3f ms per kick-drift launch" % ms, flush=True)
        return
    K, Wu = args.steps, args.warmup
    seed = w.seed + 7919 * rank
    Lf = w.leapfrog_steps
    # L2 flush buffer (larger than the 126 MB L2), written between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    total_ms, C, k_ms, k_ms_hot, launches = time_steps(P, w, prec, K, Wu, seed, barrier, flush,
                                                       fused=args.fused_trajectory, tc_grid=args.tc_grid)
    clk = clocks.stop()
    if dist is not None:
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    evals = float(C) * Lf * K * world
    value = evals / (total_ms / 1e3)

    # dominant kernel: the fused leapfrog gradient launch (kick-drift), timed
    # live with CUDA events as 20 back-to-back launches on the library's
    # stream; timed on its own at rest it is set against the burst peak, and
    # timed right after the long run of steps against the sustained one
    fl = flops_per_grad_eval(w) * C
    pk, pk_kind = peaks()
    if prec == P.FP32_SIMT:
        pkv = FP32_SIMT_PEAK_TFLOPS
        roof = {"bound": "alu", "peak": pkv, "unit": "TFLOP/s",
                "peak_source": "FP32 CUDA-core peak from unit counts at the 2032 MHz maximum clock"}
    else:
        ratio = 1.0 if prec == P.BF16 else 0.5
        pkv = pk.get("bf16_tflops", 1800.0) * ratio
        roof = {"bound": "tensor", "peak": pkv, "unit": "TFLOP/s",
                "peak_source": "%s burst bf16 (cuBLAS, maximum clock) x %.1f, for a launch timed on its own"
                               % (pk_kind, ratio)}
    roof["achieved"] = fl / (k_ms / 1e3) / 1e12
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_of(w.name, args.precision)
    roof["kernel"] = ("fused leapfrog gradient launch (kick-drift), 20 launches back to back, "
                      "before the timed steps after 1 s at rest")
    roof["kernel_ms"] = k_ms
    if prec != P.FP32_SIMT:
        pks = pk.get("bf16_tflops_sustained", 1400.0) * ratio
        a_hot = fl / (k_ms_hot / 1e3) / 1e12
        roof["after_steps"] = {"kernel_ms": k_ms_hot, "achieved": a_hot, "peak": pks, "frac": a_hot / pks,
                               "peak_source": "%s sustained bf16 (cuBLAS, 4 s loop) x %.1f" % (pk_kind, ratio)}
    roof["flops_per_launch"] = fl
    # the whole step against the same peak: L_f gradient evaluations per step
    roof["step_achieved"] = Lf * fl / (total_ms / K / 1e3) / 1e12
    roof["step_frac"] = roof["step_achieved"] / roof["peak"]

    # end to end through the C ABI with host buffers, right after the timed
    # steps (before the FP32 form's leg, which brings the power cap in):
    # create (H2D of X, y, folds), set positions (H2D), K iterations, scores
    # + diagnostics (D2H)
    theta0 = np.zeros((C, w.dim))
    truth = w.truth.get("beta", w.truth.get("phi"))
    if truth is not None:
        theta0[:, :len(truth)] = truth
    barrier()
    t0 = time.perf_counter()
    pe = P.PCV.from_workload(w, seed=seed, batch_size=K // 2 if K % 2 == 0 else 1,
                             max_batches=K + 64, acov_max_lag=64, precision=prec, init_scale=0.1)
    pe.set_positions(theta0, step_size=1e-3)
    pe.sample(K)
    sc = pe.scores()
    dg = pe.diagnostics()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    pe.close()
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())

    # the plain FP32 form on the same GPU, same workload (a few steps)
    fp32_form = None
    if prec != P.FP32_SIMT and not args.no_fp32_form:
        K32 = max(1, min(K, 3))
        ms32, _, k32, _, _ = time_steps(P, w, P.FP32_SIMT, K32, 3, seed, barrier, flush, nvtx=False)
        v32 = float(C) * Lf * K32 * world / (ms32 / 1e3)
        fp32_form = {"value": v32, "unit": "grad-evals/s", "steps": K32, "ms_per_step": ms32 / K32,
                     "kernel_ms": k32, "speedup_of_this_run": value / v32}

    h2d = 4 * w.N * w.p + 4 * w.N + 4 * w.N + 8 * C * w.dim
    d2h = 8 * w.K * 2 + 8 * 3 + 8 * w.K * 5 + 8 * 2
    _ = (sc, dg)

    line = {
        "metric": "leapfrog grad-evals/s over all fold-chains",
        "value": value, "unit": "grad-evals/s", "n_gpus": world, "steps": K, "warmup": Wu,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[args.precision],
        "data": "synthetic",
        "config": bench_config(w, args),
        # our kernels in the timed region, counted by the library (kernel
        # nodes of the iteration graphs x replays), summed over the ranks
        "gpu_launches": launches * world,
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": evals / e2e_s,
                "unit": "grad-evals/s", "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K},
    }
    if fp32_form is not None:
        line["fp32_form"] = fp32_form
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, desc, cores = oracle_rate(w, 12.0, 64 if w.N * w.p < 1e6 else 16, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": r, "unit": "grad-evals/s", "cores": cores,
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
