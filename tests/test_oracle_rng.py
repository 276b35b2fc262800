"""Pins of the oracle's counter-based RNG (Philox-4x32-10) and its transforms.

The paper draws its numbers from a per-thread Hybrid Tausworthe generator and
checks 512 streams x 10^4 draws for auto- and cross-correlations (Sec. 4.2, RNG
paragraph).  Here the generator is Philox-4x32-10 (Salmon et al. SC'11), pinned
by the published Random123 known-answer vectors, and the paper's correlation
experiment is re-run on our counter layout.
"""
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    out = oracle.philox4x32_10(ctr, key)
    assert [int(v) for v in out] == expect


def test_uniform_open_interval_and_resolution():
    lo = oracle.u01(0, 0)
    hi = oracle.u01(0xFFFFFFFF, 0xFFFFFFFF)
    assert lo == 2.0 ** -53
    assert hi == 1.0 - 2.0 ** -53
    assert 0.0 < lo < hi < 1.0
    # the low 6 bits of each word are dropped; resolution 2^-52
    assert oracle.u01(0, 63) == lo
    assert oracle.u01(63, 0) == lo
    assert oracle.u01(0, 64) == 3.0 * 2.0 ** -53
    assert oracle.u01(64, 0) == (2.0 ** 26 + 0.5) * 2.0 ** -52


def test_paper_correlation_experiment():
    """512 streams x 10^4 draws (Sec. 4.2): lag-0 cross- and lagged auto-
    correlations.  For independent streams each estimate has sd 1/sqrt(10^4) =
    0.01, so among 130816 stream pairs a few exceed 0.04 by chance (rate 6.3e-5);
    we require the exceedance rate to match that binomial expectation and no
    estimate to pass 0.05 (5 sd)."""
    U = oracle.fill_site_uniforms(1234, 0, 0, 512, 0, 10000)
    Z = U - U.mean(axis=1, keepdims=True)
    Z /= Z.std(axis=1, keepdims=True)
    C = Z @ Z.T / Z.shape[1]
    off = np.abs(C[~np.eye(512, dtype=bool)])
    n_pairs = off.size
    p_exceed = 6.334e-5  # P(|N(0, 0.01^2)| > 0.04)
    expected = n_pairs * p_exceed
    assert np.sum(off > 0.04) <= expected + 4.0 * np.sqrt(expected) + 1
    assert off.max() < 0.05
    for lag in (1, 2, 3, 10, 100):
        ac = np.mean(Z[:, lag:] * Z[:, :-lag], axis=1)
        assert np.abs(ac).max() < 0.05
        assert np.sum(np.abs(ac) > 0.04) <= 3
    np.testing.assert_allclose(np.diag(C), 1.0, atol=1e-12)


def test_uniform_chi_square():
    U = oracle.fill_site_uniforms(99, 3, 17, 64, 1000, 4000).ravel()
    counts, _ = np.histogram(U, bins=100, range=(0.0, 1.0))
    e = U.size / 100
    chi2 = np.sum((counts - e) ** 2 / e)
    # chi2 with 99 dof: mean 99, sd 14; 5 sd bound
    assert chi2 < 99 + 5 * 14


def test_box_muller_normals():
    z = []
    for n in range(4000):
        zz, _ = oracle.site_draws(7, 0, 5, n, 4)
        z.append(zz)
    z = np.array(z).ravel()
    se = 1.0 / np.sqrt(z.size)
    assert abs(z.mean()) < 4 * se
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0) * se
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3.0) < 4 * np.sqrt(24.0) * se


def test_draws_distinct_across_keys_and_counters():
    base, ub = oracle.site_draws(1, 0, 0, 0, 4)
    for args in [(2, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 0, 0, 1)]:
        z, u = oracle.site_draws(*args, 4)
        assert not np.allclose(z, base)
        assert u != ub
    zp, up = oracle.param_draws(1, 0, 0, 0)
    assert up != ub
    # a draw depends on nothing but its counter and key
    z2, u2 = oracle.site_draws(1, 0, 0, 0, 4)
    assert np.array_equal(z2, base) and u2 == ub
