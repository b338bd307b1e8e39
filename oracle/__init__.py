"""FP64 CPU oracle for PCV -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or calls it, and it imports nothing from
the product.  The C source ``pcv_oracle.c`` is compiled by ``build()`` into
``oracle/_build/liboracle.so``.

Parity status of each function (pins live in ``tests/test_oracle_*.py``):

* Philox4x32-10 -- pinned by the generator's published known-answer vectors.
* normals / uniforms / init index -- pinned by moments and exact integer math.
* log density, gradient, held-out log predictive -- pinned by conjugate
  sufficient-statistic identities, central finite differences and brute
  force sums.
* leapfrog trajectory -- pinned by the closed-form linear map on a quadratic
  potential, reversibility and O(eps^2) energy error.
* online accumulators and estimators -- pinned against two-pass batch
  formulas (eq. bmean / bmvar / rhat) on stored draws, against the AR(1)
  closed-form ESS, and against the conjugate closed-form fold posteriors.
* R-hat_max shuffle benchmark -- pinned by the identity picks (the fold's
  R-hat from stored draws), by brute-force enumeration of every pick pattern
  on a tiny case, by the uniformity of the picks, and by the paper's
  pathological chains (a shifted chain lies outside the benchmark).
* covariate-selection mask and pairwise comparison -- pinned by the
  conjugate closed form of the sub-design model (its fold elpd within MCSE)
  and of the difference of two models, and by scipy's normal cdf.
* full-data warm-up adaptation (dual averaging, mass windows) -- pinned by
  Hoffman & Gelman's closed form of the dual-averaging iterate and of its
  average, closed-loop convergence to the acceptance target on a known
  acceptance curve, numpy's sample variance over exactly the two window
  ranges of known draws (and the restart from the current step), and the
  exact full-data posterior variances of the conjugate Gaussian model.
"""
from .oracle import (  # noqa: F401
    build, lib, Problem, problem_from_workload, philox, normals, uniform,
    index, log_density, trajectory, accumulate_series, adapt_trace, shuffle_series, rhat_from_picks, compare,
    OraclePCV,
    FOLD_FIELDS, TOTAL_FIELDS,
)
