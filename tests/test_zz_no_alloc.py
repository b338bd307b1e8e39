"""GPU test of pcv_log_density_noalloc, the allocation-free gradient entry.

It serves callers that must not allocate device memory while they run (a
process whose GPU memory is owned by another framework's pool, or a
latency-bound loop where an allocation could block or synchronise the
device).  The test calls it through the C ABI twice in a row and checks both
results against the allocating pcv_log_density within the parity tolerances
of the GPU tests (log density |d|/max(|ref|,1) <= 1e-5, gradient
||d||/||ref|| <= 1e-5), checks that no allocation went through torch's
caching allocator (which the library uses as its device allocator), and that
a size beyond the fixed scratch is rejected.

This file is collected last on purpose (see the file name)."""
import ctypes as ct

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


def _rel_scalar(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1.0)


def _rel_vec(a, b):
    return np.linalg.norm(a - b, axis=-1) / np.maximum(np.linalg.norm(b, axis=-1), 1e-30)


@pytest.mark.parametrize("name", ["logistic", "hier"])
def test_noalloc_matches_allocating_entry_twice(torch, name):
    from paper_2310_07002_b300.pcv import PCV, OK, FP32_SIMT
    w = {"logistic": W.logistic_loo(N=1037, p=20, K=25, L=3),
         "hier": W.hier_logo(G=23, p=10, L=3, mean_extra=12.0)}[name]
    pc = PCV.from_workload(w)
    L = pc._L
    n = 5 * (w.K + 1) + 3
    th = torch.tensor(W.random_theta(w.dim, n, scale=0.3, seed=23), dtype=torch.float32,
                      device="cuda")
    fold = torch.tensor(np.arange(n) % (w.K + 1), dtype=torch.int32, device="cuda")
    ref_lp, ref_g, ref_sh = [t.cpu().double().numpy() for t in pc.log_density(th, fold)]
    outs = []
    for _ in range(2):
        lp = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        sh = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        g = torch.full((n, w.dim), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        st = L.pcv_log_density_noalloc(pc.h, th.data_ptr(), fold.data_ptr(), n, FP32_SIMT,
                                       lp.data_ptr(), g.data_ptr(), sh.data_ptr())
        assert st == OK, L.pcv_last_error(pc.h)
        torch.cuda.synchronize()
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == before
        outs.append([t.cpu().double().numpy() for t in (lp, g, sh)])
    for lp, g, sh in outs:
        assert _rel_scalar(lp, ref_lp).max() <= 1e-5
        assert _rel_scalar(sh, ref_sh).max() <= 1e-5
        assert _rel_vec(g, ref_g).max() <= 1e-5
    pc.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    from paper_2310_07002_b300.pcv import PCV, E_INVALID_ARG, FP32_SIMT
    w = W.logistic_loo(N=300, p=20, K=10, L=2)
    pc = PCV.from_workload(w)
    n = 8192 * 32 + 1                      # one tile more than the ticket array holds
    th = torch.zeros((n, w.dim), dtype=torch.float32, device="cuda")
    fold = torch.zeros(n, dtype=torch.int32, device="cuda")
    lp = torch.empty(n, dtype=torch.float64, device="cuda")
    sh = torch.empty(n, dtype=torch.float64, device="cuda")
    g = torch.empty((n, w.dim), dtype=torch.float32, device="cuda")
    st = pc._L.pcv_log_density_noalloc(pc.h, th.data_ptr(), fold.data_ptr(), n, FP32_SIMT,
                                       lp.data_ptr(), g.data_ptr(), sh.data_ptr())
    assert st == E_INVALID_ARG
    assert b"exceed the fixed scratch" in pc._L.pcv_last_error(pc.h)
    pc.close()
