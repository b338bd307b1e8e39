"""Pins for the oracle's leapfrog trajectory and HMC transition.

* On a quadratic potential (conjugate Gaussian model) the leapfrog map is
  linear; its closed form is the product of the kick/drift shear matrices,
  applied here with numpy matrix products.
* Reversibility: integrating back with negated momentum recovers the start.
* Energy error of the (second-order) leapfrog scales as eps^2.
"""
import numpy as np

from paper_2310_07002_b300 import workloads as W


def quad_form(w, k):
    """Precision A and linear term b of the fold-k log posterior of the
    conjugate Gaussian model: log pi = const - theta'A theta/2 + b'theta."""
    train = w.fold != k
    Xt = w.X[train]
    A = Xt.T @ Xt / w.sigma_known ** 2 + np.eye(w.p) / w.beta_prior_sd ** 2
    b = Xt.T @ w.y[train] / w.sigma_known ** 2
    return A, b


def test_leapfrog_closed_form_on_quadratic(orc):
    w = W.gauss_blocks()
    prob = orc.problem_from_workload(w)
    k, eps, Lf, p = 3, 0.05, 16, w.p
    A, b = quad_form(w, k)
    minv = np.linspace(0.5, 1.5, p)
    rng = np.random.Generator(np.random.Philox(1))
    th0 = rng.standard_normal(p)
    r0 = rng.standard_normal(p)
    # affine map on z = (theta, r, 1)
    def kick(h):
        T = np.eye(2 * p + 1)
        T[p:2 * p, :p] = -h * A
        T[p:2 * p, 2 * p] = h * b
        return T
    drift = np.eye(2 * p + 1)
    drift[:p, p:2 * p] = eps * np.diag(minv)
    T = kick(0.5 * eps)
    for s in range(1, Lf + 1):
        T = drift @ T
        T = kick(0.5 * eps if s == Lf else eps) @ T
    z = T @ np.concatenate([th0, r0, [1.0]])
    g0 = b - A @ th0
    th, r, g, lp, sh = orc.trajectory(prob, k, eps, Lf, minv, th0, r0, g0)
    assert np.allclose(th, z[:p], rtol=0, atol=1e-10)
    assert np.allclose(r, z[p:2 * p], rtol=0, atol=1e-9)
    assert np.allclose(g, b - A @ th, atol=1e-9)


def test_reversibility(orc):
    w = W.logistic_loo(N=200, p=5, K=10, L=2)
    prob = orc.problem_from_workload(w)
    minv = np.full(w.dim, 0.7)
    th0 = np.array([0.1, -0.2, 0.3, 0.05, -0.1])
    r0 = np.array([0.5, -1.0, 0.2, 0.9, -0.3])
    _, g0, _ = orc.log_density(prob, 2, th0)
    th1, r1, g1, _, _ = orc.trajectory(prob, 2, 0.03, 16, minv, th0, r0, g0)
    th2, r2, _, _, _ = orc.trajectory(prob, 2, 0.03, 16, minv, th1, -r1, g1)
    assert np.allclose(th2, th0, atol=1e-12)
    assert np.allclose(-r2, r0, atol=1e-12)


def test_energy_error_second_order(orc):
    w = W.logistic_loo(N=200, p=5, K=10, L=2)
    prob = orc.problem_from_workload(w)
    minv = np.ones(w.dim)
    th0 = np.array([0.1, -0.2, 0.3, 0.05, -0.1])
    r0 = np.array([0.5, -1.0, 0.2, 0.9, -0.3])
    lp0, g0, _ = orc.log_density(prob, 2, th0)
    H0 = -lp0 + 0.5 * r0 @ r0
    errs = []
    T = 0.32                      # fixed trajectory length
    for Lf in [8, 16, 32, 64]:
        th, r, g, lp, _ = orc.trajectory(prob, 2, T / Lf, Lf, minv, th0, r0, g0)
        errs.append(abs(-lp + 0.5 * r @ r - H0))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 3.0) & (ratios < 5.5)), ratios
