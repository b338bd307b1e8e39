"""Seeded synthetic inputs shaped like the paper's PCV workloads.

This module only *generates data* (design matrices, responses, fold
assignments).  It contains none of the method's arithmetic: no log
densities, no HMC, no estimators.  Both the FP64 oracle tests and the CUDA
path draw their inputs from here, so the two sides always see identical
bytes.

Every generator uses numpy's Philox bit generator with an explicit seed
(data seed = 1000 + workload number), so a workload is a pure function of
its arguments.

Workloads (the paper's real datasets are not available; these stand in):

* ``gauss_blocks``   -- Gaussian linear regression, contiguous K-fold blocks
                         (the conjugate case with closed-form fold posteriors).
* ``logistic_loo``   -- Bayesian logistic regression, leave-one-out.
* ``hier_logo``      -- varying-intercept Gaussian regression with uneven
                         groups, leave-one-group-out (cf. Example 1 and the
                         radon / rats examples of Section 5).
* ``ar2_hvblock``    -- AR(2) conditional regression with h(v)-block folds
                         (cf. the air-passenger time-series example).
* ``logistic_large`` -- large logistic regression with random-block folds,
                         design matrix rounded to bfloat16.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

# model kinds (values match the C ABI enum pcv_model_kind)
GAUSS_LINEAR = 0
LOGISTIC = 1
HIER_GAUSS = 2
AR_GAUSS = 3


@dataclass
class Workload:
    name: str
    kind: int
    X: np.ndarray            # float64 [N, p] row-major
    y: np.ndarray            # float64 [N]
    fold: np.ndarray         # int32 [N]; fold id 0..K-1, or -1 = in no test set
    K: int
    chains_per_fold: int
    beta_prior_sd: float
    sigma_known: float = -1.0      # > 0: known noise sd; <= 0: sampled
    sigma_prior_sd: float = 1.0
    tau_prior_sd: float = 1.0
    group: Optional[np.ndarray] = None   # int32 [N] (hierarchical only)
    n_groups: int = 0
    hv_buffer: int = 0
    leapfrog_steps: int = 16
    step_size: float = -1.0          # <= 0: adapted in the full-data warmup
    n_fulldata_warmup: int = 500
    n_fold_warmup: int = 500
    n_draws: int = 1000
    batch_size: int = 50
    seed: int = 0                    # sampler seed
    truth: dict = field(default_factory=dict)
    active: Optional[np.ndarray] = None   # int32 [p] covariate-selection mask (None: all)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def p(self) -> int:
        return int(self.X.shape[1])

    @property
    def dim(self) -> int:
        """Dimension of the unconstrained parameter vector theta."""
        if self.kind == LOGISTIC:
            return self.p
        if self.kind == HIER_GAUSS:
            return self.p + self.n_groups + 2
        return self.p + (0 if self.sigma_known > 0 else 1)

    @property
    def n_chains(self) -> int:
        return self.K * self.chains_per_fold


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (round-to-nearest-even),
    returned as float64 so every consumer reads the same rounded values."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _fp32(a: np.ndarray) -> np.ndarray:
    """Values representable in float32 (the library stores X and y in FP32),
    kept as float64 so the FP64 oracle reads exactly the GPU's inputs."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def gauss_blocks(N: int = 200, p: int = 5, K: int = 10, L: int = 4,
                 seed: int = 1001, bf16: bool = False) -> Workload:
    """Conjugate Gaussian linear regression, sigma = 1 known, beta ~ N(0, 10^2 I),
    K contiguous blocks held out.  Sampler: eps = 0.05, 16 leapfrog steps,
    identity mass, 500 warmup + 1000 draws.  bf16=True rounds X to bfloat16
    values (y is drawn from the rounded X)."""
    g = _rng(seed)
    X = g.standard_normal((N, p))
    if bf16:
        X = round_to_bf16(X)
    beta = g.standard_normal(p)
    y = X @ beta + g.standard_normal(N)
    fold = (np.arange(N) * K // N).astype(np.int32)
    X, y = _fp32(X), _fp32(y)
    return Workload("gauss_blocks", GAUSS_LINEAR, X, y, fold, K, L,
                    beta_prior_sd=10.0, sigma_known=1.0, leapfrog_steps=16,
                    step_size=0.05, n_fulldata_warmup=500, n_fold_warmup=500,
                    n_draws=1000, seed=2001, truth={"beta": beta})


def logistic_loo(N: int = 2000, p: int = 20, L: int = 8, seed: int = 1002,
                 K: Optional[int] = None, bf16: bool = False) -> Workload:
    """Logistic regression, leave-one-out (K = N folds, or the first K rows
    held out one at a time when K < N).  beta_true ~ N(0, 0.5^2),
    prior beta ~ N(0, 2.5^2 I).  bf16=True rounds X to bfloat16 values."""
    g = _rng(seed)
    X = g.standard_normal((N, p))
    if bf16:
        X = round_to_bf16(X)
    beta = 0.5 * g.standard_normal(p)
    y = (g.random(N) < _sigmoid(X @ beta)).astype(np.float64)
    K = N if K is None else K
    fold = np.full(N, -1, np.int32)
    fold[:K] = np.arange(K, dtype=np.int32)
    X = _fp32(X)
    return Workload("logistic_loo", LOGISTIC, X, y, fold, K, L,
                    beta_prior_sd=2.5, n_fulldata_warmup=500, n_fold_warmup=500,
                    n_draws=1000, seed=2002, truth={"beta": beta})


def hier_logo(G: int = 100, p: int = 10, L: int = 16, mean_extra: float = 30.0,
              seed: int = 1003, noise_p: int = 0) -> Workload:
    """Varying-intercept Gaussian model, non-centred alpha_g = tau * z_g,
    group sizes 5 + Poisson(30), leave-one-group-out.  True tau, sigma, beta,
    z drawn from the priors (tau, sigma ~ half-N(0,1), beta ~ N(0, I)).
    4000 draws: with data this informative the non-centred (tau, z) posterior
    is a ridge that a diagonal mass crosses slowly (autocorrelation time ~30
    iterations), and R-hat < 1.01 in every fold needs ~100 effective draws
    per chain.  noise_p > 0 appends that many N(0, 1) columns with true
    coefficient 0, drawn after y (the rest of the data is unchanged): a
    model with them and one without are close (a model-selection case)."""
    g = _rng(seed)
    sizes = 5 + g.poisson(mean_extra, G)
    group = np.repeat(np.arange(G, dtype=np.int32), sizes)
    N = int(sizes.sum())
    X = g.standard_normal((N, p))
    beta = g.standard_normal(p)
    tau = abs(g.standard_normal())
    sigma = abs(g.standard_normal())
    z = g.standard_normal(G)
    y = X @ beta + tau * z[group] + sigma * g.standard_normal(N)
    if noise_p > 0:
        X = np.hstack([X, g.standard_normal((N, noise_p))])
        beta = np.concatenate([beta, np.zeros(noise_p)])
    X, y = _fp32(X), _fp32(y)
    return Workload("hier_logo", HIER_GAUSS, X, y, group.copy(), G, L,
                    beta_prior_sd=1.0, sigma_prior_sd=1.0, tau_prior_sd=1.0,
                    group=group, n_groups=G, n_fulldata_warmup=500,
                    n_fold_warmup=500, n_draws=4000, seed=2003,
                    truth={"beta": beta, "tau": tau, "sigma": sigma, "z": z})


def ar2_hvblock(T: int = 5000, K: int = 250, v: int = 10, h: int = 10,
                L: int = 8, bf16: bool = False, seed: int = 1004) -> Workload:
    """AR(2) series y_t = 0.5 y_{t-1} - 0.3 y_{t-2} + e_t, e_t ~ N(0,1), 100
    burn-in values discarded.  Rows t = 3..T form the conditional regression
    on the lagged design [y_{t-1}, y_{t-2}] (N = T - 2).  Fold k tests rows
    [20k+5, 20k+15) (v = 10) and additionally excludes h rows on each side
    from its training set.  Priors phi ~ N(0, 1), sigma ~ half-N(0, 1)."""
    g = _rng(seed)
    burn = 100
    e = g.standard_normal(T + burn)
    s = np.zeros(T + burn)
    for t in range(2, T + burn):
        s[t] = 0.5 * s[t - 1] - 0.3 * s[t - 2] + e[t]
    s = s[burn:]
    y = s[2:].copy()
    X = np.stack([s[1:-1], s[:-2]], axis=1)
    if bf16:
        X = round_to_bf16(X)
    N = y.shape[0]
    fold = np.full(N, -1, np.int32)
    stride = 2 * v
    for k in range(K):
        lo = stride * k + v // 2
        hi = min(lo + v, N)
        if lo < N:
            fold[lo:hi] = k
    X, y = _fp32(X), _fp32(y)
    return Workload("ar2_hvblock", AR_GAUSS, X, y, fold, K, L,
                    beta_prior_sd=1.0, sigma_known=-1.0, sigma_prior_sd=1.0,
                    hv_buffer=h, n_fulldata_warmup=500, n_fold_warmup=500,
                    n_draws=1000, seed=2004, truth={"phi": np.array([0.5, -0.3])})


def logistic_large(N: int = 100_000, p: int = 100, K: int = 1000,
                   block: int = 100, L: int = 16, seed: int = 1005) -> Workload:
    """Large logistic regression, x_ij ~ N(0,1) rounded to bfloat16,
    beta_true ~ N(0, 0.2^2), prior beta ~ N(0, 2.5^2 I).  Random-block CV:
    a random permutation of the rows is cut into K blocks of `block` rows;
    the remaining rows are in no test set.  1000 warmup + 2000 draws."""
    g = _rng(seed)
    X = round_to_bf16(g.standard_normal((N, p)))
    beta = 0.2 * g.standard_normal(p)
    y = (g.random(N) < _sigmoid(X @ beta)).astype(np.float64)
    perm = g.permutation(N)
    fold = np.full(N, -1, np.int32)
    for k in range(K):
        fold[perm[k * block:(k + 1) * block]] = k
    return Workload("logistic_large", LOGISTIC, X, y, fold, K, L,
                    beta_prior_sd=2.5, n_fulldata_warmup=500,
                    n_fold_warmup=1000, n_draws=2000, seed=2005,
                    truth={"beta": beta})


def random_theta(dim: int, n_chains: int, scale: float = 0.3,
                 seed: int = 7) -> np.ndarray:
    """Seeded parameter vectors for single-evaluation parity tests."""
    return scale * _rng(seed).standard_normal((n_chains, dim))


def random_shat_series(n_chains: int, n_draws: int, rho: float = 0.5,
                       loc: float = -20.0, scale: float = 1.5,
                       seed: int = 11) -> np.ndarray:
    """Seeded AR(1) series standing in for held-out log predictive draws,
    used to drive the online accumulators with a known input sequence."""
    g = _rng(seed)
    e = g.standard_normal((n_chains, n_draws))
    x = np.empty_like(e)
    x[:, 0] = e[:, 0] / np.sqrt(1.0 - rho * rho)
    for t in range(1, n_draws):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return loc + scale * x


WORKLOADS = {
    "gauss_blocks": gauss_blocks,
    "logistic_loo": logistic_loo,
    "hier_logo": hier_logo,
    "ar2_hvblock": ar2_hvblock,
    "logistic_large": logistic_large,
}
