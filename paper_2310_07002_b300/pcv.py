"""Thin Python binding of the PCV C ABI (include/pcv.h).

Argument marshalling only: every step of the method runs in the CUDA
library ``_lib/libpcv.so``.  torch supplies device memory (through the
context's allocator callback and for the test entry points' buffers) and
streams.  There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libpcv.so")

# pcv_status
OK, E_INVALID_ARG, E_BAD_STATE, E_CUDA, E_OOM, E_NUMERIC, E_TIMEOUT, E_UNSUPPORTED = range(8)
STATUS_NAMES = ["OK", "INVALID_ARG", "BAD_STATE", "CUDA", "OOM", "NUMERIC", "TIMEOUT", "UNSUPPORTED"]
# pcv_model_kind
GAUSS_LINEAR, LOGISTIC, HIER_GAUSS, AR_GAUSS = range(4)
# pcv_precision
FP32_SIMT, TF32, BF16 = range(3)
PRECISIONS = {"fp32": FP32_SIMT, "tf32": TF32, "bf16": BF16}


class PCVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))


class Model(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("beta_prior_sd", ct.c_double),
                ("sigma_known", ct.c_double), ("sigma_prior_sd", ct.c_double),
                ("tau_prior_sd", ct.c_double), ("group", ct.c_void_p),
                ("n_groups", ct.c_int32), ("active_covariates", ct.c_void_p),
                ("active_covariates_b", ct.c_void_p)]


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p)


class Options(ct.Structure):
    _fields_ = [("seed", ct.c_uint64), ("leapfrog_steps", ct.c_int32),
                ("step_size", ct.c_double), ("inv_mass_diag", ct.c_void_p),
                ("batch_size", ct.c_int32), ("hv_buffer", ct.c_int32),
                ("precision", ct.c_int32), ("cuda_stream", ct.c_void_p),
                ("store_draws", ct.c_int32), ("acov_max_lag", ct.c_int32),
                ("max_batches", ct.c_int32), ("n_fulldata_draws", ct.c_int32),
                ("init_scale", ct.c_double), ("use_graphs", ct.c_int32),
                ("device_alloc", ALLOC_FN), ("device_free", FREE_FN),
                ("alloc_user", ct.c_void_p), ("trajectory_length", ct.c_double),
                ("step_jitter", ct.c_double), ("autotune", ct.c_int32),
                ("extra_scores", ct.c_int32), ("first_fold", ct.c_int32),
                ("fused_trajectory", ct.c_int32),
                ("tc_steps_per_launch", ct.c_int32),
                ("tc_grid", ct.c_int32)]


_lib = None
_D = ct.POINTER(ct.c_double)


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libpcv.so (build it first with paper_2310_07002_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError("PCV CUDA library not built: %s is missing "
                           "(run python -m paper_2310_07002_b300.build)" % _LIB_PATH)
    L = ct.CDLL(_LIB_PATH)
    vp, i32, i64, u32, f64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_uint32, ct.c_double
    sig = {
        "pcv_default_options": (None, [ct.POINTER(Options)]),
        "pcv_create": (i32, [ct.POINTER(Model), vp, vp, vp, i64, i32, i32, ct.POINTER(Options),
                             ct.POINTER(vp)]),
        "pcv_warmup": (i32, [vp, i32, i32]),
        "pcv_sample": (i32, [vp, i32]),
        "pcv_scores": (i32, [vp, vp, vp, vp, vp, vp]),
        "pcv_diagnostics": (i32, [vp, vp, vp, vp, vp, vp, vp, vp]),
        "pcv_num_folds": (i32, [vp]),
        "pcv_num_chains": (i32, [vp]),
        "pcv_dim": (i32, [vp]),
        "pcv_last_error": (ct.c_char_p, [vp]),
        "pcv_tuning_info": (i32, [vp, ct.c_char_p, i32]),
        "pcv_rhat_shuffle": (i32, [vp, i32, i32, vp, vp]),
        "pcv_compare": (i32, [vp, vp, vp, vp, vp]),
        "pcv_compare_pair": (i32, [vp, vp, vp, vp]),
        "pcv_kernel_launches": (i32, [vp, vp]),
        "pcv_scores_extra": (i32, [vp, vp, vp, vp, vp]),
        "pcv_checkpoint_size": (i32, [vp, ct.POINTER(i64)]),
        "pcv_checkpoint_save": (i32, [vp, vp, i64]),
        "pcv_checkpoint_load": (i32, [vp, vp, i64]),
        "pcv_destroy": (None, [vp]),
        "pcv_set_positions": (i32, [vp, vp, f64, vp]),
        "pcv_get_positions": (i32, [vp, vp, vp, vp]),
        "pcv_get_adaptation": (i32, [vp, vp, vp]),
        "pcv_log_density": (i32, [vp, vp, vp, i32, i32, vp, vp, vp]),
        "pcv_trajectory": (i32, [vp, vp, vp, i32, vp, vp, vp, vp]),
        "pcv_draw_normals": (i32, [vp, u32, u32, vp]),
        "pcv_accumulate": (i32, [vp, vp, i32]),
        "pcv_get_draws": (i32, [vp, vp, ct.POINTER(i32)]),
        "pcv_accept_rate": (i32, [vp, vp]),
        "pcv_last_sample_ms": (i32, [vp, ct.POINTER(f64)]),
        "pcv_setup_ms": (i32, [vp, ct.POINTER(f64), ct.POINTER(f64)]),
        "pcv_time_leapfrog_kernel": (i32, [vp, i32, ct.POINTER(f64)]),
        "pcv_log_density_noalloc": (i32, [vp, vp, vp, i32, i32, vp, vp, vp]),
        "pcv_get_pool": (i32, [vp, vp, ct.POINTER(i32)]),
        "pcv_adapt_trace": (i32, [vp, i32, vp, vp, f64, i32, vp, vp, ct.POINTER(f64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the C ABI functions this binding expects the library to export."""
    return ["pcv_default_options", "pcv_create", "pcv_warmup", "pcv_sample", "pcv_scores",
            "pcv_diagnostics", "pcv_num_folds", "pcv_num_chains", "pcv_dim", "pcv_last_error",
            "pcv_destroy", "pcv_set_positions", "pcv_get_positions", "pcv_get_adaptation",
            "pcv_log_density", "pcv_trajectory", "pcv_draw_normals", "pcv_accumulate",
            "pcv_get_draws", "pcv_accept_rate", "pcv_last_sample_ms",
            "pcv_time_leapfrog_kernel", "pcv_log_density_noalloc", "pcv_tuning_info",
            "pcv_checkpoint_size", "pcv_checkpoint_save", "pcv_checkpoint_load",
            "pcv_rhat_shuffle", "pcv_compare", "pcv_compare_pair", "pcv_kernel_launches", "pcv_scores_extra", "pcv_setup_ms",
            "pcv_get_pool", "pcv_adapt_trace"]


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _dev(t):
    """Device pointer of a contiguous CUDA tensor."""
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
    return t.data_ptr()


class _TorchAllocator:
    """Routes the library's device allocations to torch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self.device = device
        self._torch = torch

        def _alloc(nbytes, user):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device)
            except Exception:  # an allocation failure is reported as OOM by the library
                return None

        def _free(ptr, user):
            self._torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class PCV:
    """One PCV run: K folds x L chains of lock-step HMC on one GPU.

    Mirrors the C ABI: create (constructor) -> warmup -> sample* ->
    scores / diagnostics.
    """

    def __init__(self, kind: int, X, y, fold, chains_per_fold: int, *,
                 beta_prior_sd: float = 1.0, sigma_known: float = -1.0,
                 sigma_prior_sd: float = 1.0, tau_prior_sd: float = 1.0,
                 group=None, n_groups: int = 0, seed: int = 0,
                 leapfrog_steps: int = 16, step_size: float = -1.0,
                 inv_mass_diag=None, batch_size: int = 50, hv_buffer: int = 0,
                 precision: int = FP32_SIMT, stream=None, store_draws: int = 0,
                 acov_max_lag: int = 64, max_batches: int = 1024,
                 n_fulldata_draws: int = 250, init_scale: float = 1.0,
                 use_graphs: bool = True, torch_allocator: bool = True,
                 trajectory_length: float = -1.0, step_jitter: float = -1.0,
                 autotune: bool = True, active=None, extra_scores: int = 0,
                 first_fold: int = 0, fused_trajectory: int = -1, active_b=None,
                 tc_steps_per_launch: int = 0, tc_grid: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("PCV needs a CUDA device (sm_103a); none is available")
        L = load()
        self._L = L
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        fold = np.ascontiguousarray(fold, dtype=np.int32)
        self._group = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
        N, p = X.shape
        self.N, self.p, self.L = N, p, chains_per_fold
        self._active = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
        # a second model in the same launches (a subset of the covariates):
        # folds [K, 2K) and chains [K L, 2 K L) are its
        self._active_b = None if active_b is None else np.ascontiguousarray(active_b, dtype=np.int32)
        m = Model(kind, beta_prior_sd, sigma_known, sigma_prior_sd, tau_prior_sd,
                  _ptr(self._group), n_groups, _ptr(self._active), _ptr(self._active_b))
        o = Options()
        L.pcv_default_options(ct.byref(o))
        o.seed = seed
        o.leapfrog_steps = leapfrog_steps
        o.step_size = step_size
        self._minv = None if inv_mass_diag is None else np.ascontiguousarray(inv_mass_diag, dtype=np.float64)
        o.inv_mass_diag = _ptr(self._minv)
        o.batch_size = batch_size
        o.hv_buffer = hv_buffer
        o.precision = precision
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        o.cuda_stream = stream.cuda_stream
        o.store_draws = store_draws
        o.acov_max_lag = acov_max_lag
        o.max_batches = max_batches
        o.n_fulldata_draws = n_fulldata_draws
        o.init_scale = init_scale
        o.use_graphs = 1 if use_graphs else 0
        o.trajectory_length = trajectory_length
        o.step_jitter = step_jitter
        o.autotune = 1 if autotune else 0
        o.extra_scores = extra_scores
        o.first_fold = first_fold
        o.fused_trajectory = fused_trajectory
        o.tc_steps_per_launch = tc_steps_per_launch
        o.tc_grid = tc_grid
        self._alloc = None
        if torch_allocator:
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            o.device_alloc = self._alloc.alloc_fn
            o.device_free = self._alloc.free_fn
        self.batch_size = batch_size
        h = ct.c_void_p()
        st = L.pcv_create(ct.byref(m), _ptr(X), _ptr(y), _ptr(fold), N, p, chains_per_fold,
                          ct.byref(o), ct.byref(h))
        if st != OK:
            raise PCVError(st, "pcv_create: %s" % L.pcv_last_error(None).decode())
        self.h = h
        self.K = L.pcv_num_folds(h)
        self.C = L.pcv_num_chains(h)
        self.dim = L.pcv_dim(h)

    @classmethod
    def from_workload(cls, w, **kw):
        args = dict(beta_prior_sd=w.beta_prior_sd, sigma_known=w.sigma_known,
                    sigma_prior_sd=w.sigma_prior_sd, tau_prior_sd=w.tau_prior_sd,
                    group=w.group, n_groups=w.n_groups, seed=w.seed, active=w.active,
                    leapfrog_steps=w.leapfrog_steps, step_size=w.step_size,
                    batch_size=w.batch_size, hv_buffer=w.hv_buffer)
        args.update(kw)
        return cls(w.kind, w.X, w.y, w.fold, w.chains_per_fold, **args)

    def _check(self, st, what):
        if st != OK:
            msg = self._L.pcv_last_error(self.h).decode()
            raise PCVError(st, "%s: %s" % (what, msg))

    def close(self):
        if getattr(self, "h", None):
            self._L.pcv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- workflow ---------------------------------------------------------
    def warmup(self, n_fulldata_warmup: int, n_fold_warmup: int):
        self._check(self._L.pcv_warmup(self.h, n_fulldata_warmup, n_fold_warmup), "pcv_warmup")

    def sample(self, n_draws: int):
        self._check(self._L.pcv_sample(self.h, n_draws), "pcv_sample")

    def scores(self):
        e = np.empty(self.K)
        m = np.empty(self.K)
        et, mt, se = ct.c_double(), ct.c_double(), ct.c_double()
        self._check(self._L.pcv_scores(self.h, _ptr(e), _ptr(m), ct.addressof(et),
                                       ct.addressof(mt), ct.addressof(se)), "pcv_scores")
        return {"elpd": e, "mcse": m, "elpd_total": et.value, "mcse_total": mt.value,
                "se_epistemic": se.value}

    def diagnostics(self):
        K = self.K
        r, sr, eb, ea = np.empty(K), np.empty(K), np.empty(K), np.empty(K)
        dv = np.empty(K, dtype=np.int64)
        rm, et = ct.c_double(), ct.c_double()
        self._check(self._L.pcv_diagnostics(self.h, _ptr(r), _ptr(sr), _ptr(eb), _ptr(ea),
                                            _ptr(dv), ct.addressof(rm), ct.addressof(et)),
                    "pcv_diagnostics")
        return {"rhat": r, "split_rhat": sr, "ess_bm": eb, "ess_acov": ea,
                "divergences": dv, "rhat_max": rm.value, "ess_total": et.value}

    def accept_rate(self):
        a = np.empty(self.K)
        self._check(self._L.pcv_accept_rate(self.h, _ptr(a)), "pcv_accept_rate")
        return a

    def last_sample_ms(self) -> float:
        v = ct.c_double()
        self._check(self._L.pcv_last_sample_ms(self.h, ct.byref(v)), "pcv_last_sample_ms")
        return v.value

    def time_leapfrog_kernel(self, reps: int = 20) -> float:
        """Mean device milliseconds of one fused leapfrog gradient launch."""
        v = ct.c_double()
        self._check(self._L.pcv_time_leapfrog_kernel(self.h, reps, ct.byref(v)),
                    "pcv_time_leapfrog_kernel")
        return v.value

    # -- inspection / test entry points ----------------------------------
    def set_positions(self, theta, step_size: float = -1.0, inv_mass_diag=None):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        assert th.shape == (self.C, self.dim)
        mv = None if inv_mass_diag is None else np.ascontiguousarray(inv_mass_diag, dtype=np.float64)
        self._check(self._L.pcv_set_positions(self.h, _ptr(th), step_size, _ptr(mv)),
                    "pcv_set_positions")

    def positions(self):
        th = np.empty((self.C, self.dim))
        lp = np.empty(self.C)
        sh = np.empty(self.C)
        self._check(self._L.pcv_get_positions(self.h, _ptr(th), _ptr(lp), _ptr(sh)),
                    "pcv_get_positions")
        return th, lp, sh

    def scores_extra(self):
        """Hyvarinen and Dawid-Sebastiani scores (Algorithms A3, A4): per
        fold arrays and totals (NaN for a score that was not enabled)."""
        hs = np.full(self.K, np.nan)
        dss = np.full(self.K, np.nan)
        th, td = ct.c_double(), ct.c_double()
        self._check(self._L.pcv_scores_extra(self.h, _ptr(hs), _ptr(dss), ct.addressof(th),
                                             ct.addressof(td)), "pcv_scores_extra")
        return {"hs": hs, "dss": dss, "hs_total": th.value, "dss_total": td.value}

    def compare(self, other: "PCV"):
        """This model (A) against `other` (B) on the same folds (eq. sel-cv,
        norm-approx, mc-var)."""
        dk = np.empty(self.K)
        mk = np.empty(self.K)
        out = np.empty(4)
        self._check(self._L.pcv_compare(self.h, other.h, _ptr(dk), _ptr(mk), _ptr(out)), "pcv_compare")
        return {"delta_k": dk, "mcse_k": mk, "delta": out[0], "se": out[1], "mcse": out[2],
                "prob": out[3]}

    def kernel_launches(self) -> int:
        """Kernels issued by the iterations so far (graph kernel nodes x replays)."""
        n = ct.c_int64()
        self._check(self._L.pcv_kernel_launches(self.h, ct.byref(n)), "pcv_kernel_launches")
        return n.value

    def compare_pair(self):
        """Model A (folds [0, K/2)) against model B (folds [K/2, K)) of a
        context created with active_b: the same outputs as compare()."""
        K = self.K // 2
        dk = np.empty(K)
        mk = np.empty(K)
        out = np.empty(4)
        self._check(self._L.pcv_compare_pair(self.h, _ptr(dk), _ptr(mk), _ptr(out)), "pcv_compare_pair")
        return {"delta_k": dk, "mcse_k": mk, "delta": out[0], "se": out[1], "mcse": out[2],
                "prob": out[3]}

    def rhat_shuffle(self, n_blocks: int = 5, n_reps: int = 500, per_fold: bool = False):
        """R-hat_max benchmark replicates (Section 4.2): [n_reps] maxima over
        folds, and [n_reps, K] per-fold values when per_fold."""
        mx = np.empty(n_reps)
        allv = np.empty((n_reps, self.K)) if per_fold else None
        self._check(self._L.pcv_rhat_shuffle(self.h, n_blocks, n_reps, _ptr(mx), _ptr(allv)),
                    "pcv_rhat_shuffle")
        return (mx, allv) if per_fold else mx

    def checkpoint(self) -> bytes:
        """The run's state as bytes (see pcv_checkpoint_save)."""
        n = ct.c_int64()
        self._check(self._L.pcv_checkpoint_size(self.h, ct.byref(n)), "pcv_checkpoint_size")
        buf = ct.create_string_buffer(n.value)
        self._check(self._L.pcv_checkpoint_save(self.h, buf, n.value), "pcv_checkpoint_save")
        return buf.raw

    def restore(self, blob: bytes):
        """Continue a run from checkpoint() bytes (same model, data and options)."""
        buf = ct.create_string_buffer(blob, len(blob))
        self._check(self._L.pcv_checkpoint_load(self.h, buf, len(blob)), "pcv_checkpoint_load")

    def tuning_info(self) -> str:
        buf = ct.create_string_buffer(4096)
        self._check(self._L.pcv_tuning_info(self.h, buf, len(buf)), "pcv_tuning_info")
        return buf.value.decode()

    def setup_ms(self):
        """Host milliseconds spent so far in the autotuner and in CUDA-graph
        capture (both inside warmup / sample, reported apart)."""
        a, g = ct.c_double(), ct.c_double()
        self._check(self._L.pcv_setup_ms(self.h, ct.byref(a), ct.byref(g)), "pcv_setup_ms")
        return {"autotune_ms": a.value, "graph_capture_ms": g.value}

    def adaptation(self):
        e = ct.c_double()
        mv = np.empty(self.dim)
        self._check(self._L.pcv_get_adaptation(self.h, ct.addressof(e), _ptr(mv)),
                    "pcv_get_adaptation")
        return e.value, mv

    def pool(self):
        """The full-data draws the fold chains start from, [4 n_keep, dim]."""
        n = ct.c_int32()
        self._check(self._L.pcv_get_pool(self.h, None, ct.byref(n)), "pcv_get_pool")
        out = np.empty((n.value, self.dim))
        self._check(self._L.pcv_get_pool(self.h, _ptr(out), ct.byref(n)), "pcv_get_pool")
        return out

    def adapt_trace(self, accept, draws, eps0: float = 0.1, adapt_mass: bool = True):
        """The full-data adaptation on given inputs (accept [n, 4], draws
        [n, 4, dim] as float32): step size and inverse mass after each
        iteration, and the final dual-averaged step size (no cap)."""
        acc = np.ascontiguousarray(accept, dtype=np.float64)
        dr = np.ascontiguousarray(draws, dtype=np.float32)
        n = acc.shape[0]
        assert acc.shape == (n, 4) and dr.shape == (n, 4, self.dim)
        eps = np.empty(n)
        minv = np.empty((n, self.dim))
        fin = ct.c_double()
        self._check(self._L.pcv_adapt_trace(self.h, n, _ptr(acc), _ptr(dr), eps0, int(adapt_mass),
                                            _ptr(eps), _ptr(minv), ct.byref(fin)), "pcv_adapt_trace")
        return eps, minv, fin.value

    def log_density(self, theta, fold, precision: int = FP32_SIMT):
        """(logp [n] f64, grad [n, dim] f32, shat [n] f64) for CUDA tensors
        theta [n, dim] f32 and fold [n] int32 (K = full data)."""
        import torch
        n = theta.shape[0]
        logp = torch.empty(n, dtype=torch.float64, device=theta.device)
        shat = torch.empty(n, dtype=torch.float64, device=theta.device)
        grad = torch.empty_like(theta)
        self._check(self._L.pcv_log_density(self.h, _dev(theta), _dev(fold), n, precision,
                                            _dev(logp), _dev(grad), _dev(shat)),
                    "pcv_log_density")
        return logp, grad, shat

    def trajectory(self, theta0, r0, precision: int = FP32_SIMT):
        import torch
        th1 = torch.empty_like(theta0)
        r1 = torch.empty_like(r0)
        lp = torch.empty(self.C, dtype=torch.float64, device=theta0.device)
        sh = torch.empty(self.C, dtype=torch.float64, device=theta0.device)
        self._check(self._L.pcv_trajectory(self.h, _dev(theta0), _dev(r0), precision,
                                           _dev(th1), _dev(r1), _dev(lp), _dev(sh)),
                    "pcv_trajectory")
        return th1, r1, lp, sh

    def draw_normals(self, iteration: int, stream: int = 0):
        import torch
        out = torch.empty((self.C, self.dim), dtype=torch.float32, device="cuda")
        self._check(self._L.pcv_draw_normals(self.h, iteration, stream, _dev(out)),
                    "pcv_draw_normals")
        return out

    def accumulate(self, shat):
        self._check(self._L.pcv_accumulate(self.h, _dev(shat), shat.shape[1]), "pcv_accumulate")

    def draws(self):
        n = ct.c_int32()
        self._check(self._L.pcv_get_draws(self.h, None, ct.byref(n)), "pcv_get_draws")
        out = np.empty((self.C, n.value))
        self._check(self._L.pcv_get_draws(self.h, _ptr(out), ct.byref(n)), "pcv_get_draws")
        return out


def _masked_log_density_fn():
    import torch

    class MaskedLogDensity(torch.autograd.Function):
        """log pi_k(theta) for a batch of (theta, fold) pairs with the
        hand-written gradient kernel as its backward (eq. mask-log-prob)."""

        @staticmethod
        def forward(ctx, theta, pcv: PCV, fold, precision: int = FP32_SIMT):
            th = theta.detach().to(torch.float32).contiguous()
            logp, grad, _ = pcv.log_density(th, fold, precision)
            ctx.save_for_backward(grad)
            return logp

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return (g.to(grad.dtype)[:, None] * grad, None, None, None)

    return MaskedLogDensity


_MLD = None


def masked_log_density(theta, pcv: PCV, fold, precision: int = FP32_SIMT):
    global _MLD
    if _MLD is None:
        _MLD = _masked_log_density_fn()
    return _MLD.apply(theta, pcv, fold, precision)
