"""Multi-process (gloo, CPU) test of the fold-range sharding host logic: two
ranks each own half of the folds, compute their fold results (here with the
oracle on a given draw series), gather and merge; the merged per-fold results
equal a single-process run exactly and the totals to rounding."""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2310_07002_b300 import shard
from paper_2310_07002_b300 import workloads as W


def test_fold_ranges_partition_the_folds():
    for K, world in [(10, 2), (7, 3), (1000, 8), (5, 5)]:
        rs = [shard.fold_range(K, world, r) for r in range(world)]
        assert rs[0][0] == 0 and rs[-1][1] == K
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [b - a for a, b in rs]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.fold_range(3, 4, 0)


def test_shard_folds_renumbers_and_releases_other_rows():
    fold = np.array([0, 1, 2, 3, -1, 2, 1, 0], np.int32)
    out = shard.shard_folds(fold, 1, 3)
    assert out.tolist() == [-1, 0, 1, -1, -1, 1, 0, -1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, path_s, path_out, L, b, M):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = np.load(path_s)
    K = s.shape[0] // L
    k0, k1 = shard.fold_range(K, world, rank)
    fo, _ = oracle.accumulate_series(s[k0 * L:k1 * L], L, b, M)
    local = {k: fo[k] for k in ("elpd", "mcse", "rhat", "split_rhat", "ess_bm", "ess_acov", "divergences")}
    merged = shard.merge(shard.gather(local))
    if rank == 0:
        np.save(path_out, np.array([merged], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_single_run(orc):
    import torch.multiprocessing as mp
    L, b, M, K = 4, 25, 8, 9
    s = W.random_shat_series(K * L, 400, rho=0.5, loc=-30.0, scale=2.0, seed=17)
    s[5] += 0.7
    with tempfile.TemporaryDirectory() as td:
        ps, po = os.path.join(td, "s.npy"), os.path.join(td, "out.npy")
        np.save(ps, s)
        mp.start_processes(_worker, args=(2, _free_port(), ps, po, L, b, M), nprocs=2, join=True,
                           start_method="spawn")
        merged = np.load(po, allow_pickle=True)[0]
    fo, to = orc.accumulate_series(s, L, b, M)
    for k in ("elpd", "mcse", "rhat", "split_rhat", "ess_bm", "ess_acov"):
        assert np.array_equal(merged[k], fo[k]), k
    assert abs(merged["elpd_total"] - to["elpd"]) < 1e-9
    assert abs(merged["mcse_total"] - to["mcse"]) < 1e-12
    assert abs(merged["se_epistemic"] - to["se_epistemic"]) < 1e-9
    assert merged["rhat_max"] == to["rhat_max"]
