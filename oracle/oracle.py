"""ctypes binding of the FP64 oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

FOLD_FIELDS = ["elpd", "mcse", "sig2_bm_rel", "s2_rel", "ess_bm", "rhat",
               "split_rhat", "ess_acov", "divergences", "acov_truncated",
               "accept_rate"]
TOTAL_FIELDS = ["elpd", "mcse", "se_epistemic", "rhat_max", "ess_total",
                "split_rhat_max", "divergences"]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        _declare(_lib)
    return _lib


class Problem(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("p", ct.c_int32), ("N", ct.c_int64),
                ("X", ct.c_void_p), ("y", ct.c_void_p), ("fold", ct.c_void_p),
                ("K", ct.c_int32), ("h", ct.c_int32), ("group", ct.c_void_p),
                ("G", ct.c_int32), ("beta_sd", ct.c_double),
                ("sigma_known", ct.c_double), ("sigma_sd", ct.c_double),
                ("tau_sd", ct.c_double), ("active", ct.c_void_p)]


_D = ct.POINTER(ct.c_double)
_U32 = ct.POINTER(ct.c_uint32)


def _declare(L):
    L.orc_philox.argtypes = [_U32, _U32, _U32]
    L.orc_normals.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32, ct.c_int32, _D]
    L.orc_uniform.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32]
    L.orc_uniform.restype = ct.c_double
    L.orc_index.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32, ct.c_uint32]
    L.orc_index.restype = ct.c_uint32
    L.orc_dim.argtypes = [ct.POINTER(Problem)]
    L.orc_dim.restype = ct.c_int32
    L.orc_log_density.argtypes = [ct.POINTER(Problem), ct.c_int32, _D, _D, _D, _D]
    L.orc_log_density.restype = ct.c_int
    L.orc_trajectory.argtypes = [ct.POINTER(Problem), ct.c_int32, ct.c_double, ct.c_int32,
                                 _D, _D, _D, _D, _D, _D]
    L.orc_trajectory.restype = ct.c_int
    L.orc_accumulate_series.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, _D, ct.c_int32,
                                        ct.c_int32, ct.c_int32, _D, _D]
    L.orc_accumulate_series.restype = ct.c_int
    L.orc_pcv_create.argtypes = [ct.POINTER(Problem), ct.c_int32, ct.c_uint64, ct.c_int32,
                                 ct.c_double, _D, ct.c_int32, ct.c_int32, ct.c_int32,
                                 ct.c_int32, ct.c_int32, ct.c_double]
    L.orc_pcv_create.restype = ct.c_void_p
    L.orc_pcv_destroy.argtypes = [ct.c_void_p]
    _I = ct.POINTER(ct.c_int32)
    L.orc_shuffle_series.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, _D, ct.c_int32, ct.c_int32,
                                     ct.c_int32, ct.c_int32, ct.c_uint64, _D, _D]
    L.orc_shuffle_series.restype = ct.c_int
    L.orc_rhat_from_picks_series.argtypes = [ct.c_int32, ct.c_int32, _D, ct.c_int32, ct.c_int32, _I, _D]
    L.orc_rhat_from_picks_series.restype = ct.c_int
    L.orc_pcv_rhat_shuffle.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _D]
    L.orc_pcv_rhat_shuffle.restype = ct.c_int
    L.orc_pcv_enable_extra.argtypes = [ct.c_void_p, ct.c_int32]
    L.orc_pcv_enable_extra.restype = ct.c_int
    L.orc_pcv_extra_results.argtypes = [ct.c_void_p, _D, _D]
    L.orc_pcv_extra_results.restype = ct.c_int
    L.orc_compare.argtypes = [ct.c_int32, _D, _D, _D, _D, _D, _D, _D]
    L.orc_compare.restype = ct.c_int
    L.orc_pcv_set_tuning.argtypes = [ct.c_void_p, ct.c_double, ct.c_double]
    L.orc_pcv_set_tuning.restype = ct.c_int
    L.orc_pcv_set_chain_base.argtypes = [ct.c_void_p, ct.c_int64]
    L.orc_pcv_set_chain_base.restype = ct.c_int
    L.orc_pcv_fulldata.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_double]
    L.orc_pcv_fulldata.restype = ct.c_int
    L.orc_pcv_fulldata_accept.argtypes = [ct.c_void_p, _D, _D]
    L.orc_pcv_fulldata_accept.restype = ct.c_int
    L.orc_adapt_trace.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, _D, _D, ct.c_double, ct.c_int32,
                                  ct.c_int32, _D, ct.POINTER(ct.c_int32), ct.c_int32, _D, _D, _D]
    L.orc_adapt_trace.restype = ct.c_int
    L.orc_pcv_fold_warmup.argtypes = [ct.c_void_p, ct.c_int32]
    L.orc_pcv_fold_warmup.restype = ct.c_int
    L.orc_pcv_set_state.argtypes = [ct.c_void_p, _D, ct.c_double, _D]
    L.orc_pcv_set_state.restype = ct.c_int
    L.orc_pcv_sample.argtypes = [ct.c_void_p, ct.c_int32]
    L.orc_pcv_sample.restype = ct.c_int
    L.orc_pcv_results.argtypes = [ct.c_void_p, _D, _D]
    L.orc_pcv_results.restype = ct.c_int
    L.orc_pcv_get_draws.argtypes = [ct.c_void_p, _D]
    L.orc_pcv_get_draws.restype = ct.c_int
    L.orc_pcv_get_state.argtypes = [ct.c_void_p, _D, _D, _D, _D, _D]
    L.orc_pcv_get_state.restype = ct.c_int
    L.orc_pcv_theta_stats.argtypes = [ct.c_void_p, _D, _D, _D]
    L.orc_pcv_theta_stats.restype = ct.c_int
    L.orc_pcv_get_pool.argtypes = [ct.c_void_p, _D, ct.POINTER(ct.c_int32)]
    L.orc_pcv_get_pool.restype = ct.c_int


def _dp(a: Optional[np.ndarray]):
    if a is None:
        return ct.cast(None, _D)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


class _ProblemHolder:
    """Keeps the numpy arrays behind a Problem struct alive."""

    def __init__(self, kind, X, y, fold, K, h=0, group=None, G=0, beta_sd=1.0,
                 sigma_known=-1.0, sigma_sd=1.0, tau_sd=1.0, active=None):
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.fold = np.ascontiguousarray(fold, dtype=np.int32)
        self.group = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
        self.active = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
        N, p = self.X.shape
        self.s = Problem(kind, p, N, self.X.ctypes.data, self.y.ctypes.data,
                         self.fold.ctypes.data, K, h,
                         None if self.group is None else self.group.ctypes.data,
                         G, beta_sd, sigma_known, sigma_sd, tau_sd,
                         None if self.active is None else self.active.ctypes.data)

    @property
    def dim(self) -> int:
        return int(lib().orc_dim(ct.byref(self.s)))


def problem_from_workload(w) -> _ProblemHolder:
    return _ProblemHolder(w.kind, w.X, w.y, w.fold, w.K, w.hv_buffer, w.group,
                          w.n_groups, w.beta_prior_sd, w.sigma_known,
                          w.sigma_prior_sd, w.tau_prior_sd, w.active)


def compare(elpd_a, mcse_a, elpd_b, mcse_b):
    """Pairwise model selection (eq. sel-cv, norm-approx, mc-var): returns a
    dict with delta_k, mcse_k, delta, se, mcse, prob (Pr(A better than B))."""
    ea, ma, eb, mb = (np.ascontiguousarray(v, dtype=np.float64) for v in (elpd_a, mcse_a, elpd_b, mcse_b))
    K = ea.size
    dk = np.empty(K)
    mk = np.empty(K)
    out = np.empty(4)
    assert lib().orc_compare(K, _dp(ea), _dp(ma), _dp(eb), _dp(mb), _dp(dk), _dp(mk), _dp(out)) == 0
    return {"delta_k": dk, "mcse_k": mk, "delta": out[0], "se": out[1], "mcse": out[2], "prob": out[3]}


def adapt_trace(accept, draws, eps0=0.1, adapt_eps=True, adapt_mass=True, minv0=None,
                active=None):
    """The full-data warm-up adaptation (Section 3.1) driven by given inputs:
    accept[i] is the chains' mean acceptance statistic after iteration i and
    draws[i, c, :] the position of chain c after it.  Returns (step size after
    each iteration [n], inverse mass after each iteration [n, d], final step
    size with no cap)."""
    acc = np.ascontiguousarray(accept, dtype=np.float64)
    dr = np.ascontiguousarray(draws, dtype=np.float64)
    n, nc, d = dr.shape
    assert acc.shape == (n,)
    m0 = np.ones(d) if minv0 is None else np.ascontiguousarray(minv0, dtype=np.float64)
    act = None if active is None else np.ascontiguousarray(active, dtype=np.int32)
    eps = np.empty(n)
    minv = np.empty((n, d))
    fin = ct.c_double()
    rc = lib().orc_adapt_trace(n, nc, d, _dp(acc), _dp(dr), eps0, int(adapt_eps), int(adapt_mass), _dp(m0),
                               None if act is None else act.ctypes.data_as(ct.POINTER(ct.c_int32)),
                               0 if act is None else act.size, _dp(eps), _dp(minv), ct.byref(fin))
    assert rc == 0
    return eps, minv, fin.value


def philox(ctr, key):
    c = (ct.c_uint32 * 4)(*ctr)
    k = (ct.c_uint32 * 2)(*key)
    o = (ct.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return list(o)


def normals(seed, chain, it, stream, n):
    z = np.empty(n)
    lib().orc_normals(seed, chain, it, stream, n, _dp(z))
    return z


def uniform(seed, chain, it, stream):
    return lib().orc_uniform(seed, chain, it, stream)


def index(seed, chain, it, stream, n):
    return lib().orc_index(seed, chain, it, stream, n)


def log_density(prob: _ProblemHolder, fold_id: int, theta: np.ndarray):
    """(logp, grad, shat) at theta for fold `fold_id` (-1: full data)."""
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    g = np.empty(prob.dim)
    lp = ct.c_double()
    sh = ct.c_double()
    rc = lib().orc_log_density(ct.byref(prob.s), fold_id, _dp(theta),
                               ct.byref(lp), _dp(g), ct.byref(sh))
    assert rc == 0
    return lp.value, g, sh.value


def trajectory(prob, fold_id, eps, Lf, minv, theta, r, grad):
    th = np.array(theta, dtype=np.float64)
    rr = np.array(r, dtype=np.float64)
    gg = np.array(grad, dtype=np.float64)
    mv = np.ascontiguousarray(minv, dtype=np.float64)
    lp = ct.c_double()
    sh = ct.c_double()
    rc = lib().orc_trajectory(ct.byref(prob.s), fold_id, eps, Lf, _dp(mv), _dp(th),
                              _dp(rr), _dp(gg), ct.byref(lp), ct.byref(sh))
    assert rc == 0
    return th, rr, gg, lp.value, sh.value


def accumulate_series(s: np.ndarray, L: int, b: int, M: int = 64,
                      max_batches: int = 4096):
    """Run a given draw sequence s[C, n] through the online accumulators.
    Returns (fold results dict of arrays, totals dict)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    C, n = s.shape
    K = C // L
    fo = np.empty((K, len(FOLD_FIELDS)))
    to = np.empty(len(TOTAL_FIELDS))
    rc = lib().orc_accumulate_series(C, L, n, _dp(s), b, M, max_batches, _dp(fo), _dp(to))
    assert rc == 0
    return ({f: fo[:, i] for i, f in enumerate(FOLD_FIELDS)},
            {f: to[i] for i, f in enumerate(TOTAL_FIELDS)})


def shuffle_series(s: np.ndarray, L: int, b: int, D: int, R: int, seed: int,
                   max_batches: int = 4096):
    """R-hat_max benchmark (Section 4.2) on a given draw sequence s[C, n]:
    returns (R-hat_max of each replicate [R], per-fold values [R, K])."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    C, n = s.shape
    out = np.empty(R)
    allv = np.empty((R, C // L))
    rc = lib().orc_shuffle_series(C, L, n, _dp(s), b, max_batches, D, R, seed, _dp(out), _dp(allv))
    assert rc == 0
    return out, allv


def rhat_from_picks(s: np.ndarray, b: int, D: int, picks) -> float:
    """R-hat of L chains rebuilt from blocks: block d of slot l comes from
    chain picks[l][d] (s[L, n])."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    L, n = s.shape
    pk = np.ascontiguousarray(np.asarray(picks, dtype=np.int32).reshape(L * D))
    out = np.empty(1)
    rc = lib().orc_rhat_from_picks_series(L, n, _dp(s), b, D,
                                          pk.ctypes.data_as(ct.POINTER(ct.c_int32)), _dp(out))
    assert rc == 0
    return float(out[0])


class OraclePCV:
    """A whole PCV run in the oracle: warm-up reuse, sampling, estimators."""

    def __init__(self, prob: _ProblemHolder, L: int, seed: int, Lf: int,
                 eps: float = -1.0, minv: Optional[np.ndarray] = None, b: int = 50,
                 M: int = 64, max_batches: int = 4096, store_draws: bool = False,
                 n_threads: int = 0, init_scale: float = 1.0, traj_len: float = -1.0,
                 jitter: float = -1.0, chain_base: int = 0):
        self.prob = prob
        self.L = L
        self.K = prob.s.K
        self.C = self.K * L
        self.d = prob.dim
        self._minv = None if minv is None else np.ascontiguousarray(minv, dtype=np.float64)
        nt = n_threads if n_threads > 0 else (os.cpu_count() or 1)
        self.h = lib().orc_pcv_create(ct.byref(prob.s), L, seed, Lf, eps, _dp(self._minv),
                                      b, M, max_batches, int(store_draws), nt, init_scale)
        # trajectory-length cap and step-size jitter (< 0: the defaults)
        lib().orc_pcv_set_tuning(self.h, traj_len, jitter)
        # Philox chain id of fold chain c = chain_base + c
        assert lib().orc_pcv_set_chain_base(self.h, chain_base) == 0

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_pcv_destroy(self.h)
            self.h = None

    def fulldata(self, n_adapt: int, n_keep: int, eps0: float = 0.1):
        assert lib().orc_pcv_fulldata(self.h, n_adapt, n_keep, eps0) == 0

    def fulldata_accept(self):
        """Mean acceptance statistics of the full-data chains: over the
        adaptation iterations since dual averaging last (re)started, and over
        the iterations kept in the pool (fixed settings)."""
        t = ct.c_double()
        k = ct.c_double()
        assert lib().orc_pcv_fulldata_accept(self.h, ct.byref(t), ct.byref(k)) == 0
        return t.value, k.value

    def fold_warmup(self, n_wu: int):
        assert lib().orc_pcv_fold_warmup(self.h, n_wu) == 0

    def set_state(self, theta: np.ndarray, eps: float = -1.0, minv=None):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        assert theta.shape == (self.C, self.d)
        mv = None if minv is None else np.ascontiguousarray(minv, dtype=np.float64)
        assert lib().orc_pcv_set_state(self.h, _dp(theta), eps, _dp(mv)) == 0

    def sample(self, n_draws: int):
        assert lib().orc_pcv_sample(self.h, n_draws) == 0

    def results(self):
        fo = np.empty((self.K, len(FOLD_FIELDS)))
        to = np.empty(len(TOTAL_FIELDS))
        assert lib().orc_pcv_results(self.h, _dp(fo), _dp(to)) == 0
        return ({f: fo[:, i] for i, f in enumerate(FOLD_FIELDS)},
                {f: to[i] for i, f in enumerate(TOTAL_FIELDS)})

    def enable_extra_scores(self, flags: int = 3):
        """Accumulate the Hyvarinen (1) and Dawid-Sebastiani (2) scores."""
        assert lib().orc_pcv_enable_extra(self.h, flags) == 0

    def extra_scores(self):
        hs = np.empty(self.K)
        dss = np.empty(self.K)
        assert lib().orc_pcv_extra_results(self.h, _dp(hs), _dp(dss)) == 0
        return hs, dss

    def rhat_shuffle(self, D: int, R: int):
        out = np.empty(R)
        assert lib().orc_pcv_rhat_shuffle(self.h, D, R, _dp(out)) == 0
        return out

    def draws(self, n: int):
        out = np.empty((self.C, n))
        assert lib().orc_pcv_get_draws(self.h, _dp(out)) == 0
        return out

    def state(self):
        th = np.empty((self.C, self.d))
        eps = ct.c_double()
        mv = np.empty(self.d)
        lp = np.empty(self.C)
        sh = np.empty(self.C)
        lib().orc_pcv_get_state(self.h, _dp(th), ct.byref(eps), _dp(mv), _dp(lp), _dp(sh))
        return {"theta": th, "eps": eps.value, "minv": mv, "logp": lp, "shat": sh}

    def pool(self):
        n = ct.c_int32()
        lib().orc_pcv_get_pool(self.h, None, ct.byref(n))
        out = np.empty((n.value, self.d))
        lib().orc_pcv_get_pool(self.h, _dp(out), ct.byref(n))
        return out

    def theta_stats(self):
        """Per chain: running posterior mean of theta and the Welford
        (mean, M2) of its batch means, each [C, d]."""
        m = np.empty((self.C, self.d))
        bm = np.empty((self.C, self.d))
        b2 = np.empty((self.C, self.d))
        assert lib().orc_pcv_theta_stats(self.h, _dp(m), _dp(bm), _dp(b2)) == 0
        return m, bm, b2
