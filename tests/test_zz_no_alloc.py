"""GPU tests of pcv_log_density_noalloc, the allocation-free gradient entry.

It serves callers that must not allocate device memory while they run (a
process whose GPU memory is owned by another framework's pool, or a
latency-bound loop where an allocation could block or synchronise the
device).  Through the C ABI, two calls in a row each time:
  * on FP32 contexts: against the allocating pcv_log_density and against the
    FP64 oracle, within the FP32 parity tolerances of the GPU tests (log
    density |d|/max(|ref|,1) <= 1e-5, gradient ||d||/||ref|| <= 1e-5), and
    no allocation through torch's caching allocator (the library's device
    allocator);
  * on BF16 and TF32 contexts, where the call still runs the FP32 kernel:
    against the oracle at the FP32 tolerances;
  * with 64-chain tiles (p > 32) and a request whose usual split count does
    not fit the fixed scratch, so the call runs fewer splits: against
    pcv_log_density and the oracle;
  * one request beyond each of the two fixed limits (tickets, scratch), each
    rejected with a message naming it.

This file is collected last on purpose (see the file name)."""
import numpy as np
import pytest

from paper_2310_07002_b300 import workloads as W

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 4 << 20
TICKETS = 8192
TARGET_CTAS = 148 * 4


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_07002_b300.build import build
    build()
    return torch


def _rel_scalar(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def _rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


def _noalloc(torch, pc, th, fold, check_alloc=True):
    from paper_2310_07002_b300.pcv import OK, FP32_SIMT
    n, d = th.shape
    lp = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    sh = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    g = torch.full((n, d), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    st = pc._L.pcv_log_density_noalloc(pc.h, th.data_ptr(), fold.data_ptr(), n, FP32_SIMT,
                                       lp.data_ptr(), g.data_ptr(), sh.data_ptr())
    assert st == OK, pc._L.pcv_last_error(pc.h)
    torch.cuda.synchronize()
    if check_alloc:
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
    return [t.cpu().double().numpy() for t in (lp, g, sh)]


def _against_oracle(orc, w, th, folds, out, rows):
    prob = orc.problem_from_workload(w)
    lp, g, sh = out
    for i in rows:
        k = int(folds[i])
        rl, rg, rs = orc.log_density(prob, -1 if k == w.K else k, th[i])
        assert _rel_scalar(lp[i], rl) <= 1e-5, (i, lp[i], rl)
        assert _rel_scalar(sh[i], rs) <= 1e-5, (i, sh[i], rs)
        assert _rel_vec(g[i], rg) <= 1e-5, (i, _rel_vec(g[i], rg))


def _inputs(torch, w, n, scale, seed):
    th = torch.tensor(W.random_theta(w.dim, n, scale=scale, seed=seed), dtype=torch.float32, device="cuda")
    folds = np.arange(n) % (w.K + 1)
    return th, torch.tensor(folds, dtype=torch.int32, device="cuda"), folds


@pytest.mark.parametrize("name", ["logistic", "hier"])
def test_noalloc_matches_allocating_entry_and_oracle_twice(torch, orc, name):
    from paper_2310_07002_b300.pcv import PCV
    w = {"logistic": W.logistic_loo(N=1037, p=20, K=25, L=3),
         "hier": W.hier_logo(G=23, p=10, L=3, mean_extra=12.0)}[name]
    pc = PCV.from_workload(w)
    n = 5 * (w.K + 1) + 3
    th, fold, folds = _inputs(torch, w, n, 0.3, 23)
    ref_lp, ref_g, ref_sh = [t.cpu().double().numpy() for t in pc.log_density(th, fold)]
    outs = [_noalloc(torch, pc, th, fold) for _ in range(2)]
    for lp, g, sh in outs:
        assert _rel_scalar(lp, ref_lp).max() <= 1e-5
        assert _rel_scalar(sh, ref_sh).max() <= 1e-5
        assert _rel_vec(g, ref_g).max() <= 1e-5
    thn = th.cpu().double().numpy()
    for out in outs:
        _against_oracle(orc, w, thn, folds, out, range(0, n, 7))
    pc.close()


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_noalloc_runs_fp32_on_tensor_core_contexts(torch, orc, precision):
    from paper_2310_07002_b300.pcv import PCV, PRECISIONS
    w = W.logistic_loo(N=1037, p=20, K=25, L=3, bf16=True)
    pc = PCV.from_workload(w, precision=PRECISIONS[precision])
    n = 130
    th, fold, folds = _inputs(torch, w, n, 0.3, 24)
    outs = [_noalloc(torch, pc, th, fold) for _ in range(2)]
    thn = th.cpu().double().numpy()
    for out in outs:
        _against_oracle(orc, w, thn, folds, out, range(n))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    pc.close()


def test_noalloc_wide_tiles_with_fewer_splits(torch, orc):
    from paper_2310_07002_b300.pcv import PCV
    # p = 128: 64-chain tiles, 132 partial sums per chain.  640 positions =
    # 10 tiles; the usual split count fills 4 CTAs per SM, ceil(592 / 10) =
    # 60 splits (the row cap N / 256 = 78 allows it), whose partials would
    # need 60 x 10 x 64 x 132 floats > 4 Mi: the call runs 49 splits.
    w = W.logistic_loo(N=20000, p=128, K=40, L=2)
    n, T, width = 640, 64, 128 + 4
    tiles = n // T
    usual = min(-(-TARGET_CTAS // tiles), w.N // 256)
    assert usual * tiles * T * width > SCRATCH_FLOATS
    assert SCRATCH_FLOATS // (tiles * T * width) < usual
    pc = PCV.from_workload(w)
    th, fold, folds = _inputs(torch, w, n, 0.05, 25)
    ref_lp, ref_g, ref_sh = [t.cpu().double().numpy() for t in pc.log_density(th, fold)]
    outs = [_noalloc(torch, pc, th, fold) for _ in range(2)]
    thn = th.cpu().double().numpy()
    for lp, g, sh in outs:
        assert _rel_scalar(lp, ref_lp).max() <= 1e-5
        assert _rel_scalar(sh, ref_sh).max() <= 1e-5
        assert _rel_vec(g, ref_g).max() <= 1e-5
    for out in outs:
        _against_oracle(orc, w, thn, folds, out, [0, 1, 63, 64, 127, 320, 639])
    pc.close()


@pytest.mark.parametrize("limit", ["tickets", "scratch"])
def test_noalloc_rejects_each_limit(torch, limit):
    from paper_2310_07002_b300.pcv import PCV, E_INVALID_ARG, FP32_SIMT
    if limit == "tickets":
        # p = 4: 32-chain tiles of 8 partial sums per chain; 8193 tiles fit the
        # scratch (8193 x 32 x 8 floats < 4 Mi) but not the ticket array
        w = W.gauss_blocks(N=200, p=4, K=10, L=2)
        n = (TICKETS + 1) * 32
        assert (TICKETS + 1) * 32 * 8 <= SCRATCH_FLOATS
        msg = b"ticket array"
    else:
        # p = 100: 64-chain tiles of 104 partial sums; 631 tiles (well under
        # the ticket limit) need 631 x 64 x 104 floats > 4 Mi
        w = W.logistic_loo(N=300, p=100, K=10, L=2)
        n = 631 * 64
        assert 631 * 64 * 104 > SCRATCH_FLOATS
        msg = b"fixed scratch"
    pc = PCV.from_workload(w)
    th = torch.zeros((n, w.dim), dtype=torch.float32, device="cuda")
    fold = torch.zeros(n, dtype=torch.int32, device="cuda")
    lp = torch.empty(n, dtype=torch.float64, device="cuda")
    sh = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, w.dim), dtype=torch.float32, device="cuda")
    st = pc._L.pcv_log_density_noalloc(pc.h, th.data_ptr(), fold.data_ptr(), n, FP32_SIMT,
                                       lp.data_ptr(), g.data_ptr(), sh.data_ptr())
    assert st == E_INVALID_ARG
    err = pc._L.pcv_last_error(pc.h)
    assert msg in err, err
    # one size under the limit is accepted
    ok = n - (32 if limit == "tickets" else 64)
    st = pc._L.pcv_log_density_noalloc(pc.h, th.data_ptr(), fold.data_ptr(), ok, FP32_SIMT,
                                       lp.data_ptr(), g.data_ptr(), sh.data_ptr())
    assert st == 0, pc._L.pcv_last_error(pc.h)
    torch.cuda.synchronize()
    pc.close()
