"""Fold-range sharding of one PCV problem over several GPUs.

Folds are independent posteriors (Section 3), so the path shards with no
data-path exchange: each rank owns a contiguous range of folds and runs its
own context on the full data, with the rows of the other folds marked as in
no test set (they train in every fold, as in a single-context run) and
``first_fold`` set so that its chains draw the Philox streams of the same
global folds.  The only exchange is the final gather of the K-length fold
results, merged here into the totals of eq. cv-score, eq. mc-var and
eq. norm-approx and R-hat_max (eq. rhat-max).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


def fold_range(K: int, world: int, rank: int) -> Tuple[int, int]:
    """Contiguous, balanced [k0, k1) range of global folds for `rank`."""
    if not (0 <= rank < world) or K < world:
        raise ValueError("need 0 <= rank < world <= K")
    return K * rank // world, K * (rank + 1) // world


def shard_folds(fold: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """Fold assignment of a shard: folds k0..k1-1 renumbered from 0, every
    other row in no test set (-1)."""
    fold = np.asarray(fold, dtype=np.int32)
    out = np.full(fold.shape, -1, np.int32)
    own = (fold >= k0) & (fold < k1)
    out[own] = fold[own] - k0
    return out


def local_results(pc) -> Dict[str, np.ndarray]:
    """The per-fold results of one shard's context, ready to gather."""
    sc, dg = pc.scores(), pc.diagnostics()
    return {"elpd": sc["elpd"], "mcse": sc["mcse"], "rhat": dg["rhat"],
            "split_rhat": dg["split_rhat"], "ess_bm": dg["ess_bm"], "ess_acov": dg["ess_acov"],
            "divergences": np.asarray(dg["divergences"], dtype=np.float64)}


def merge(parts: Sequence[Dict[str, np.ndarray]]) -> Dict[str, object]:
    """Concatenate the shards' fold results in rank order (global fold order)
    and form the totals: elpd = sum, MCSE = sqrt(sum MCSE_k^2) (eq. mc-var),
    se_epistemic = sqrt(K var_k(elpd_k)) (eq. norm-approx), R-hat_max."""
    cat = {k: np.concatenate([np.asarray(p[k], dtype=np.float64) for p in parts]) for k in parts[0]}
    K = cat["elpd"].size
    out: Dict[str, object] = dict(cat)
    out["elpd_total"] = float(cat["elpd"].sum())
    out["mcse_total"] = float(np.sqrt(np.sum(cat["mcse"] ** 2)))
    out["se_epistemic"] = float(np.sqrt(K * np.var(cat["elpd"], ddof=1))) if K > 1 else float("nan")
    out["rhat_max"] = float(cat["rhat"].max())
    out["split_rhat_max"] = float(np.nanmax(cat["split_rhat"]))
    out["divergences_total"] = float(cat["divergences"].sum())
    return out


def gather(local: Dict[str, np.ndarray], group=None) -> List[Dict[str, np.ndarray]]:
    """All ranks' fold results, in rank order (torch.distributed, any backend)."""
    import torch.distributed as dist
    parts: List[object] = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, {k: np.asarray(v) for k, v in local.items()}, group=group)
    return parts  # type: ignore[return-value]
