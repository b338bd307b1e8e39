"""Pins for the oracle's online accumulators and estimators (Algorithm A2,
Appendix A.1, eq. bmean, bmvar, mc-var, rhat, rhat-max, Section 4.1).

The online results must equal two-pass batch formulas written here directly
from the definitions over the same stored draws; the autocorrelation ESS is
pinned against the AR(1) closed form tau = (1 + rho) / (1 - rho); R-hat
against i.i.d. chains and the pathological stuck / shifted chains of
Section 4.2."""
import numpy as np
import pytest
from scipy.special import logsumexp

from paper_2310_07002_b300 import workloads as W


def rhat_def(chains):
    """eq. rhat for chains[L, n]."""
    L, n = chains.shape
    means = chains.mean(axis=1)
    Wv = chains.var(axis=1, ddof=1).mean()
    B = n / (L - 1) * ((means - means.mean()) ** 2).sum()
    return np.sqrt(((n - 1) / n * Wv + B / n) / Wv)


def geyer_ess(chains, M):
    """Multi-chain autocorrelation ESS with Geyer's initial monotone
    sequence, from stored draws (direct autocovariance sums)."""
    L, n = chains.shape
    means = chains.mean(axis=1)
    Wv = chains.var(axis=1, ddof=1).mean()
    B = n / (L - 1) * ((means - means.mean()) ** 2).sum()
    varplus = (n - 1) / n * Wv + B / n
    Mu = min(M, n - 1)
    rho = np.empty(Mu + 1)
    for m in range(Mu + 1):
        g = [np.sum((c[m:] - c.mean()) * (c[:n - m] - c.mean())) / n for c in chains]
        rho[m] = 1 - (Wv - np.mean(g)) / varplus
    rho[0] = 1.0
    tau, prev, trunc = -1.0, np.inf, 1
    for k in range(Mu // 2 + 1):
        if 2 * k + 1 > Mu:
            break
        P = rho[2 * k] + rho[2 * k + 1]
        if not P > 0:
            trunc = 0
            break
        P = min(P, prev)
        prev = P
        tau += 2 * P
    return L * n / tau, trunc


def batch_estimates(s, L, b, M):
    """Two-pass per-fold estimates from stored draws s[C, n]."""
    C, n = s.shape
    K = C // L
    a = n // b
    out = {f: np.empty(K) for f in ["elpd", "mcse", "sig2_bm_rel", "s2_rel", "ess_bm",
                                    "rhat", "split_rhat", "ess_acov"]}
    for k in range(K):
        sk = s[k * L:(k + 1) * L]
        f = np.exp(sk).mean()
        bm = np.exp(sk).reshape(L, a, b).mean(axis=2)          # eq. bmean
        sig2 = b / (L * a - 1) * ((bm - f) ** 2).sum()         # eq. bmvar
        s2 = ((np.exp(sk) - f) ** 2).sum() / (L * n - 1)
        out["elpd"][k] = logsumexp(sk) - np.log(L * n)
        out["sig2_bm_rel"][k] = sig2 / f ** 2
        out["s2_rel"][k] = s2 / f ** 2
        out["mcse"][k] = np.sqrt(sig2 / (L * n)) / f            # eq. mc-var
        out["ess_bm"][k] = L * n * s2 / sig2
        out["rhat"][k] = rhat_def(sk)
        half = (a // 2) * b
        halves = np.concatenate([sk[:, :half], sk[:, n - half:]], axis=0)
        out["split_rhat"][k] = rhat_def(halves)
        out["ess_acov"][k] = geyer_ess(sk, M)[0]
    return out


@pytest.mark.parametrize("n,b", [(500, 50), (550, 50), (300, 25)])
def test_online_equals_batch(orc, n, b):
    L, K, M = 4, 3, 30
    s = W.random_shat_series(K * L, n, rho=0.6, loc=-30.0, scale=2.0, seed=21)
    fo, to = orc.accumulate_series(s, L, b, M)
    ref = batch_estimates(s, L, b, M)
    for key, val in ref.items():
        assert np.allclose(fo[key], val, rtol=1e-10, atol=0), key
    assert abs(to["elpd"] - ref["elpd"].sum()) < 1e-9
    assert abs(to["mcse"] - np.sqrt((ref["mcse"] ** 2).sum())) < 1e-12
    assert abs(to["rhat_max"] - ref["rhat"].max()) < 1e-12
    ess_tot = L * n * ref["s2_rel"].sum() / ref["sig2_bm_rel"].sum()
    assert abs(to["ess_total"] / ess_tot - 1) < 1e-10
    se = np.sqrt(K * np.var(ref["elpd"], ddof=1))
    assert abs(to["se_epistemic"] - se) < 1e-10


def test_extreme_log_scale_no_underflow(orc):
    # held-out joint log densities of -2000 underflow exp() in FP64; the
    # log-shifted accumulators must still give the batch answers.
    L, K, n, b = 4, 2, 200, 50
    s = W.random_shat_series(K * L, n, rho=0.3, loc=-2000.0, scale=1.0, seed=3)
    fo, _ = orc.accumulate_series(s, L, b, 20)
    ref = batch_estimates(s - (-2000.0), L, b, 20)     # shift-invariance
    assert np.allclose(fo["elpd"], ref["elpd"] - 2000.0, rtol=1e-12)
    for key in ["mcse", "ess_bm", "rhat", "split_rhat", "ess_acov"]:
        assert np.allclose(fo[key], ref[key], rtol=1e-9), key


def test_ar1_ess_closed_form(orc):
    rho = 0.5
    L, n = 4, 40000
    s = W.random_shat_series(L, n, rho=rho, loc=-10.0, scale=0.05, seed=4)
    fo, _ = orc.accumulate_series(s, L, 100, 64)
    frac_theory = (1 - rho) / (1 + rho)
    assert abs(fo["ess_acov"][0] / (L * n) / frac_theory - 1) < 0.1
    assert abs(fo["ess_bm"][0] / (L * n) / frac_theory - 1) < 0.2


def test_rhat_iid_and_pathological(orc):
    L, K, n, b = 4, 2, 2000, 50
    g = np.random.Generator(np.random.Philox(8))
    s = -5.0 + g.standard_normal((K * L, n))
    fo, _ = orc.accumulate_series(s, L, b, 10)
    assert np.all(fo["rhat"] < 1.01) and np.all(fo["split_rhat"] < 1.01)
    stuck = s.copy()
    stuck[1, :] = stuck[1, 0]             # one chain fixed at its first draw
    fo_s, _ = orc.accumulate_series(stuck, L, b, 10)
    assert fo_s["rhat"][0] > 1.05 and fo_s["rhat"][1] == fo["rhat"][1]
    shifted = s.copy()
    shifted[5, :] += 5.0                  # one chain shifted by 5 units
    fo_h, _ = orc.accumulate_series(shifted, L, b, 10)
    assert fo_h["rhat"][1] > 1.5 and fo_h["rhat"][0] == fo["rhat"][0]
