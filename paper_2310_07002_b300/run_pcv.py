"""Run a whole parallel cross-validation on one of the synthetic workloads and
print one JSON line with the scores, the diagnostics and the wall clock of
each phase.

    python -m paper_2310_07002_b300.run_pcv --workload logistic_large \
        [--precision bf16] [--draws N] [--fd-warmup N] [--fold-warmup N] \
        [--compare fp32]

The phases are those of the PCV workflow (Section 3): create (data to the
device), warm-up (full-data adaptation, then the fold chains' discarded
warm-up; Section 3.1), sampling with the online accumulators (Algorithm A2)
and the estimators (Section 3.2, Section 4). `--compare` runs the same
workload again at a second precision with another sampler seed and reports,
per fold, z = (elpd_a - elpd_b) / sqrt(MCSE_a^2 + MCSE_b^2).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import workloads as W

WORKLOADS = {
    "gauss_blocks": lambda: W.gauss_blocks(),
    "logistic_loo": lambda: W.logistic_loo(),
    # X rounded to bf16 values: both precisions then see the same data, so a
    # comparison measures arithmetic only
    "logistic_loo_bf16x": lambda: W.logistic_loo(bf16=True),
    "hier_logo": lambda: W.hier_logo(),
    # config 3 with one pure-noise covariate appended (index 10; true
    # coefficient 0): with and without it the models are close
    "hier_logo_noise": lambda: W.hier_logo(noise_p=1),
    "ar2_hvblock": lambda: W.ar2_hvblock(),
    # lagged design rounded to bf16 values for both precisions (arithmetic only)
    "ar2_hvblock_bf16x": lambda: W.ar2_hvblock(bf16=True),
    "logistic_large": lambda: W.logistic_large(),
}


def run(w, precision: str, draws: int, fd_warmup: int, fold_warmup: int, seed: int, keep=False):
    import torch
    from . import pcv as P
    t = {}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pc = P.PCV.from_workload(w, precision=P.PRECISIONS[precision], seed=seed)
    torch.cuda.synchronize()
    t["create_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pc.warmup(fd_warmup, fold_warmup)
    torch.cuda.synchronize()
    t["warmup_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pc.sample(draws)
    torch.cuda.synchronize()
    t["sample_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sc = pc.scores()
    dg = pc.diagnostics()
    t["finalize_s"] = time.perf_counter() - t0
    # R-hat_max benchmark (Section 4.2): 500 block-shuffled replicates, 5 blocks
    t0 = time.perf_counter()
    rep = pc.rhat_shuffle(5, 500) if draws // w.batch_size >= 5 else None
    shuffle_s = time.perf_counter() - t0
    eps, _ = pc.adaptation()
    acc = pc.accept_rate()
    C = pc.C
    su = pc.setup_ms()
    if not keep:
        pc.close()
    t["total_s"] = sum(t.values())
    # one-off costs inside warm-up and sampling, stated apart (not added to
    # the total a second time)
    t["of_which_autotune_s"] = su["autotune_ms"] / 1e3
    t["of_which_graph_capture_s"] = su["graph_capture_ms"] / 1e3
    t["rhat_shuffle_benchmark_s"] = shuffle_s   # after the run, not in the total
    evals = float(C) * w.leapfrog_steps * (fold_warmup + draws)
    out = {
        "precision": precision, "seed": seed, "chains": C,
        "elpd": float(sc["elpd_total"]), "mcse": float(sc["mcse_total"]),
        "se_epistemic": float(sc["se_epistemic"]),
        "rhat_max": float(dg["rhat_max"]),
        "rhat_max_shuffle_q": (None if rep is None else
                               [float(q) for q in np.quantile(rep, [0.05, 0.5, 0.95])]),
        "rhat_max_shuffle_rank": (None if rep is None else float(np.mean(rep < dg["rhat_max"]))),
        "split_rhat_max": float(np.max(dg["split_rhat"])),
        "folds_rhat_ge_1.01": int(np.sum(dg["rhat"] >= 1.01)),
        "ess_total": float(dg["ess_total"]),
        "ess_bm_min": float(np.min(dg["ess_bm"])), "ess_acov_min": float(np.min(dg["ess_acov"])),
        "divergences": int(np.sum(dg["divergences"])),
        "accept_mean": float(np.mean(acc)), "step_size": float(eps),
        "fold_grad_evals_per_s": evals / (t["warmup_s"] + t["sample_s"]),
        "wall": t,
    }
    if keep:
        return out, sc, dg, pc
    return out, sc, dg


def pair_progress(w, precision: str, draws: int, fd_warmup: int, fold_warmup: int, seed: int,
                  drop: str, n_reports: int):
    """Models A (all covariates) and B (without `drop`) in one context: both
    models' chains in every launch (Appendix B's masks); after each of
    n_reports equal parts of the draws, the comparison (eq. sel-cv,
    norm-approx, mc-var) and the largest fold R-hat of each model."""
    import torch
    from . import pcv as P
    act = np.ones(w.p, np.int32)
    act[[int(v) for v in drop.split(",")]] = 0
    t0 = time.perf_counter()
    pc = P.PCV.from_workload(w, precision=P.PRECISIONS[precision], seed=seed, active_b=act)
    pc.warmup(fd_warmup, fold_warmup)
    torch.cuda.synchronize()
    warm_s = time.perf_counter() - t0
    K = pc.K // 2
    step = max(w.batch_size, draws // n_reports // w.batch_size * w.batch_size)
    rows, done, sample_s = [], 0, 0.0
    while done < draws:
        n = min(step, draws - done)
        t1 = time.perf_counter()
        pc.sample(n)
        torch.cuda.synchronize()
        sample_s += time.perf_counter() - t1
        done += n
        c = pc.compare_pair()
        dg = pc.diagnostics()
        rows.append({"draws": done, "delta": c["delta"], "se": c["se"], "mcse": c["mcse"],
                     "prob_a_better": c["prob"], "rhat_max_a": float(np.max(dg["rhat"][:K])),
                     "rhat_max_b": float(np.max(dg["rhat"][K:]))})
    sc = pc.scores()
    out = {"workload": w.name, "N": w.N, "p": w.p, "K": K, "L": w.chains_per_fold, "dropped": drop,
           "chains_per_launch": pc.C, "precision": precision, "seed": seed, "draws": draws,
           "fd_warmup": fd_warmup, "fold_warmup": fold_warmup,
           "elpd_a": float(np.sum(sc["elpd"][:K])), "elpd_b": float(np.sum(sc["elpd"][K:])),
           "warmup_s": warm_s, "sample_s": sample_s, "progress": rows}
    pc.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="logistic_large", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16", choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--draws", type=int, default=None)
    ap.add_argument("--fd-warmup", type=int, default=None)
    ap.add_argument("--fold-warmup", type=int, default=None)
    ap.add_argument("--compare", default=None, choices=["fp32", "tf32", "bf16"])
    ap.add_argument("--compare-draws", type=int, default=None,
                    help="draws of the comparison run (default: the same)")
    ap.add_argument("--compare-fold-warmup", type=int, default=None)
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--pair-drop", default=None,
                    help="comma-separated covariate indices: run model B (without them) in the same "
                         "launches as model A, one context, and report the comparison as sampling "
                         "proceeds (the progressive estimate of Fig. 1)")
    ap.add_argument("--progress", type=int, default=10, help="reports over the draws (--pair-drop)")
    ap.add_argument("--drop-covariates", default=None,
                    help="comma-separated covariate indices: also run model B without them "
                         "(Appendix B's selection mask) and report the pairwise comparison")
    args = ap.parse_args()
    from .build import build
    build()
    w = WORKLOADS[args.workload]()
    draws = args.draws or w.n_draws
    fdw = args.fd_warmup or w.n_fulldata_warmup
    fow = args.fold_warmup or w.n_fold_warmup
    seed = w.seed if args.seed is None else args.seed
    if args.pair_drop is not None:
        print(json.dumps(pair_progress(w, args.precision, draws, fdw, fow, seed, args.pair_drop, args.progress)),
              flush=True)
        return
    sel = args.drop_covariates is not None
    if sel:
        a, sca, dga, pa = run(w, args.precision, draws, fdw, fow, seed, keep=True)
    else:
        a, sca, dga = run(w, args.precision, draws, fdw, fow, seed)
    line = {"workload": w.name, "N": w.N, "p": w.p, "K": w.K, "L": w.chains_per_fold,
            "leapfrog_steps": w.leapfrog_steps, "draws": draws, "fd_warmup": fdw,
            "fold_warmup": fow, "batch_size": w.batch_size, "run": a}
    if args.compare:
        b, scb, dgb = run(w, args.compare, args.compare_draws or draws, fdw,
                          args.compare_fold_warmup or fow, seed + 1)
        z = (sca["elpd"] - scb["elpd"]) / np.sqrt(sca["mcse"] ** 2 + scb["mcse"] ** 2)

        def infl(sc, dg):   # batch-means MCSE inflated where ESS_bm exceeds ESS_acov
            return sc["mcse"] * np.sqrt(np.maximum(1.0, dg["ess_bm"] / dg["ess_acov"]))
        zi = (sca["elpd"] - scb["elpd"]) / np.hypot(infl(sca, dga), infl(scb, dgb))
        zt = (a["elpd"] - b["elpd"]) / np.hypot(a["mcse"], b["mcse"])
        line["compare"] = {"run": b, "z_total": float(zt), "z_abs_max": float(np.max(np.abs(z))),
                           "z_abs_mean": float(np.mean(np.abs(z))),
                           "folds_abs_z_gt_3": int(np.sum(np.abs(z) > 3)),
                           "z_acov_abs_max": float(np.max(np.abs(zi))),
                           "folds_abs_z_acov_gt_3": int(np.sum(np.abs(zi) > 3)),
                           "speedup_grad_evals": a["fold_grad_evals_per_s"] / b["fold_grad_evals_per_s"]}
    if sel:
        import dataclasses
        act = np.ones(w.p, np.int32)
        act[[int(v) for v in args.drop_covariates.split(",")]] = 0
        b_run, _, _, pb = run(dataclasses.replace(w, active=act), args.precision, draws, fdw, fow, seed, keep=True)
        t0 = time.perf_counter()
        c = pa.compare(pb)
        compare_s = time.perf_counter() - t0
        line["selection"] = {"dropped": args.drop_covariates, "model_b": b_run,
                             "delta": c["delta"], "se": c["se"], "mcse": c["mcse"],
                             "prob_a_better": c["prob"], "compare_s": compare_s}
        pa.close()
        pb.close()
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
