"""Pins of the oracle's RBE mode sampler (Sec. 2.2, Eq. 12; Algorithm 1 step 1).

  * the normaliser S (the paper's Q) against the Poisson identity
    (tests/golden/poisson_S.txt, written from the closed form alone);
  * chi-square tests of the drawn modes against the exact law
    P(m) = exp(-k^2/4alpha)/S over m != 0 (marginals and |m|^2 shells);
  * no drawn mode is m = 0, even where P(m = 0) is large.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poisson_S.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, L, S = line.split()
        rows.append((int(n), float(L), float(S)))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_S_matches_poisson_identity(row):
    _, L, S_ref = row
    S = oracle.rbe_S(L, 0.62)
    assert abs(S - S_ref) <= 1e-6 * S_ref + 1e-6


def test_M_truncation_is_below_1e16():
    for L in (17.1, 79.37, 171.0, 368.4):
        a = oracle.sampler_a(L, 0.62)
        M = oracle.sampler_M(L, 0.62)
        assert math.exp(-a * M * M) < 1e-16
        assert math.exp(-a * (M - 1) * (M - 1)) >= 1e-16 * 0.999


def _exact_marginal(L, alpha):
    M, _, H = oracle.sampler_table(L, alpha)
    a = oracle.sampler_a(L, alpha)
    m = np.arange(-M, M + 1)
    w = np.exp(-a * m * m)
    S = H ** 3 - 1.0
    p = w * (H * H - (m == 0)) / S
    return m, p


@pytest.mark.parametrize("L,alpha", [(17.1, 0.62), (4.0, 2.0)])
def test_marginals_chi_square(L, alpha):
    P = 200_000
    m = oracle.rbe_sample(seed=7, step=3, P=P, L=L, alpha=alpha)
    assert not np.any(np.all(m == 0, axis=1))
    mv, p = _exact_marginal(L, alpha)
    for d in range(3):
        obs = np.array([np.sum(m[:, d] == k) for k in mv], dtype=float)
        exp = p * P
        keep = exp >= 5
        o = np.append(obs[keep], obs[~keep].sum())
        e = np.append(exp[keep], exp[~keep].sum())
        if e[-1] < 5:
            o[-2] += o[-1]; e[-2] += e[-1]
            o, e = o[:-1], e[:-1]
        chi2 = np.sum((o - e) ** 2 / e)
        pval = stats.chi2.sf(chi2, len(o) - 1)
        assert pval > 1e-4, (d, chi2, len(o), pval)


def test_shell_distribution_chi_square():
    # Joint law: P(|m|^2 = s) = g(s) exp(-a s)/S, g = number of lattice points.
    L, alpha = 6.0, 1.0
    M, _, H = oracle.sampler_table(L, alpha)
    a = oracle.sampler_a(L, alpha)
    S = H ** 3 - 1.0
    r = np.arange(-M, M + 1)
    s = (r[:, None, None] ** 2 + r[None, :, None] ** 2 + r[None, None, :] ** 2).ravel()
    s = s[s > 0]
    smax = 12
    exp_p = np.array([np.sum(s == k) * math.exp(-a * k) / S for k in range(1, smax + 1)])
    P = 100_000
    m = oracle.rbe_sample(seed=11, step=0, P=P, L=L, alpha=alpha)
    ms = np.sum(m.astype(np.int64) ** 2, axis=1)
    obs = np.array([np.sum(ms == k) for k in range(1, smax + 1)], dtype=float)
    obs = np.append(obs, np.sum(ms > smax))
    exp = np.append(exp_p, 1 - exp_p.sum()) * P
    keep = exp > 0
    o, e = obs[keep], exp[keep]
    chi2 = np.sum((o - e) ** 2 / e)
    assert stats.chi2.sf(chi2, len(o) - 1) > 1e-4


def test_zero_mode_rejected_in_small_box():
    # L = 2, alpha = 4: P(m = 0) = 1/H^3 is about 0.04 per attempt.
    m = oracle.rbe_sample(seed=1, step=5, P=50_000, L=2.0, alpha=4.0)
    assert not np.any(np.all(m == 0, axis=1))


def test_draws_depend_on_seed_step_replica():
    a = oracle.rbe_sample(0, 0, 64, 17.1, 0.62)
    assert np.array_equal(a, oracle.rbe_sample(0, 0, 64, 17.1, 0.62))
    assert not np.array_equal(a, oracle.rbe_sample(0, 1, 64, 17.1, 0.62))
    assert not np.array_equal(a, oracle.rbe_sample(1, 0, 64, 17.1, 0.62))
    assert not np.array_equal(a, oracle.rbe_sample(0, 0, 64, 17.1, 0.62, replica=1))
