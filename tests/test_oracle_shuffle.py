"""Pins for the oracle's R-hat_max benchmark (Section 4.2; the block-shuffle
loop of Algorithm A2): chains are cut into D contiguous blocks of whole
batches and rebuilt from blocks of chains drawn with replacement; the R-hat
(eq. rhat) of the rebuilt chains, maximised over folds, gives one
replicate."""
import itertools

import numpy as np

from paper_2310_07002_b300 import workloads as W


def rhat_np(x):
    """eq. rhat from the draws themselves (two-pass)."""
    L, n = x.shape
    Wv = x.var(axis=1, ddof=1).mean()
    B = n * x.mean(axis=1).var(ddof=1)
    return np.sqrt(((n - 1) / n * Wv + B / n) / Wv)


def rebuild(x, b, D, picks):
    """Slot l, block d = block d (whole batches d a / D .. (d+1) a / D) of chain picks[l][d]."""
    L, n = x.shape
    a = n // b
    out = []
    for l in range(L):
        parts = []
        for d in range(D):
            h0, h1 = d * a // D, (d + 1) * a // D
            parts.append(x[picks[l][d], h0 * b:h1 * b])
        out.append(np.concatenate(parts))
    return np.stack(out)


def test_identity_picks_give_the_folds_rhat(orc):
    s = W.random_shat_series(4, 600, rho=0.6, seed=3)
    for D in (1, 3, 5):
        ident = [[l] * D for l in range(4)]
        assert abs(orc.rhat_from_picks(s, 20, D, ident) - rhat_np(s)) < 1e-12


def test_picked_blocks_match_brute_force_concatenation(orc):
    s = W.random_shat_series(3, 500, rho=0.4, seed=5)
    g = np.random.default_rng(1)
    for D in (2, 5, 7):                  # 7 does not divide a = 25: uneven blocks
        for _ in range(5):
            picks = g.integers(0, 3, size=(3, D))
            ref = rhat_np(rebuild(s, 20, D, picks))
            assert abs(orc.rhat_from_picks(s, 20, D, picks) - ref) < 1e-12


def test_replicates_enumerate_the_pick_patterns_uniformly(orc):
    # L = 2 chains, D = 2 blocks: 16 possible pick patterns; every replicate
    # is one of them, and each occurs with probability 1/16
    s = W.random_shat_series(2, 400, rho=0.3, seed=9)
    pats = list(itertools.product([0, 1], repeat=4))
    vals = np.array([rhat_np(rebuild(s, 10, 2, np.array(p).reshape(2, 2))) for p in pats])
    R = 3200
    mx, allv = orc.shuffle_series(s, L=2, b=10, D=2, R=R, seed=77)
    assert np.allclose(mx, allv[:, 0])
    idx = np.array([np.argmin(np.abs(vals - v)) for v in mx])
    assert np.all(np.abs(vals[idx] - mx) < 1e-12)
    # patterns with equal R-hat are merged into one class for the count
    cls = np.unique(np.round(vals, 12), return_inverse=True)[1]
    counts = np.bincount(cls[idx], minlength=cls.max() + 1)
    expect = np.bincount(cls, minlength=cls.max() + 1) * R / 16
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 40.0                    # df <= 15: p ~ 5e-4


def test_shifted_chain_lies_outside_the_benchmark(orc):
    # the paper's pathological case: one chain of one fold shifted by 5 units
    K, L, n, b = 20, 4, 1000, 50
    s = W.random_shat_series(K * L, n, rho=0.5, seed=21)
    mx, _ = orc.shuffle_series(s, L=L, b=b, D=5, R=500, seed=3)
    _, tot = orc.accumulate_series(s, L=L, b=b, M=8)
    assert tot["rhat_max"] <= np.quantile(mx, 0.995)     # mixed: inside the histogram
    s2 = s.copy()
    s2[7] += 5.0
    mx2, _ = orc.shuffle_series(s2, L=L, b=b, D=5, R=500, seed=3)
    _, tot2 = orc.accumulate_series(s2, L=L, b=b, M=8)
    assert tot2["rhat_max"] > mx2.max()
    # a stuck chain (constant at its first draw) too
    s3 = s.copy()
    s3[11] = s3[11, 0]
    mx3, _ = orc.shuffle_series(s3, L=L, b=b, D=5, R=500, seed=3)
    _, tot3 = orc.accumulate_series(s3, L=L, b=b, M=8)
    assert tot3["rhat_max"] > mx3.max()
