"""Pins for the oracle's counter-based generator (Philox4x32-10) and the
derived uniforms, normals and init indices."""
import numpy as np
import pytest
from scipy import stats

from tests.golden.load import philox_kat


def test_philox_known_answers(orc):
    rows = philox_kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert orc.philox(ctr, key) == expect


def test_uniform_is_word0_offset(orc):
    # u = (w0 + 0.5) / 2^32 on the open interval (0, 1)
    seed = 0x1234_5678_9ABC_DEF0
    for chain, it, st in [(0, 0, 1), (17, 3, 1), (4095, 123456, 17)]:
        w = orc.philox([0, chain, it, st], [seed & 0xFFFFFFFF, seed >> 32])
        u = orc.uniform(seed, chain, it, st)
        assert u == (w[0] + 0.5) / 2.0 ** 32
        assert 0.0 < u < 1.0


def test_index_exact_integer(orc):
    seed = 99
    for chain in range(50):
        w = orc.philox([0, chain, 0, 2], [seed, 0])
        n = 1000 + chain
        assert orc.index(seed, chain, 0, 2, n) == (w[0] * n) >> 32


def test_index_uniform_chi2(orc):
    n = 10
    counts = np.zeros(n)
    for chain in range(5000):
        counts[orc.index(5, chain, 0, 2, n)] += 1
    chi2 = ((counts - 500.0) ** 2 / 500.0).sum()
    assert stats.chi2.sf(chi2, n - 1) > 1e-4


def test_normals_box_muller_mapping(orc):
    # element i: Philox block i // 4; words (0,1) -> (cos, sin) pair, (2,3) next
    seed, chain, it, st = 42, 3, 7, 0
    z = orc.normals(seed, chain, it, st, 10)
    for i in range(10):
        w = orc.philox([i // 4, chain, it, st], [seed, 0])
        pr = (i % 4) // 2
        u1 = (w[2 * pr] + 0.5) / 2.0 ** 32
        u2 = (w[2 * pr + 1] + 0.5) / 2.0 ** 32
        rad = np.sqrt(-2.0 * np.log(u1))
        ref = rad * (np.cos(2 * np.pi * u2) if i % 2 == 0 else np.sin(2 * np.pi * u2))
        assert abs(z[i] - ref) < 1e-12


def test_normals_distribution(orc):
    z = np.concatenate([orc.normals(7, c, 0, 0, 100) for c in range(1000)])
    assert abs(z.mean()) < 5.0 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # pairs from one Box-Muller draw are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.03


def test_streams_independent(orc):
    a = np.concatenate([orc.normals(7, c, 0, 0, 8) for c in range(2000)])
    b = np.concatenate([orc.normals(7, c, 0, 16, 8) for c in range(2000)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.04
    assert not np.allclose(a[:8], b[:8])
