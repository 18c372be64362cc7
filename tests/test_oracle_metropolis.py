"""Pins of the oracle's Metropolis mode chains (Algorithm 1 step 1).

The chains start from the exact i.i.d. draw and satisfy detailed balance for
exp(-a |m|^2) on Z^3 \\ {0}, so at every later step the states are distributed
exactly like the i.i.d. sampler's: the marginal of m_x and the distribution of
|m|^2 are compared with the exact probabilities (summed over the lattice) by
chi-square tests.  The chains do move, and zero moves per step freezes them.
"""
import math

import numpy as np
import pytest

import oracle

L, ALPHA = 17.1, 0.62


def exact_marginal(L=L):
    a = math.pi ** 2 / (ALPHA * L * L)
    M = oracle.sampler_M(L, ALPHA)
    r = np.arange(-M, M + 1)
    w = np.exp(-a * r * r)
    H = w.sum()
    S = H ** 3 - 1.0
    # P(m_x = j) over m != 0: w_j (H^2 - [j == 0]) / S
    p = w * (H * H - (r == 0)) / S
    return r, p


def chi2_pvalue(counts, expected):
    from scipy import stats

    keep = expected >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(expected[keep], expected[~keep].sum())
    if exp[-1] < 5:
        obs, exp = obs[:-1], exp[:-1]
    c2 = float(np.sum((obs - exp) ** 2 / exp))
    return stats.chi2.sf(c2, len(obs) - 1)


@pytest.mark.parametrize("box,step,moves,P", [(L, 0, 8, 20000), (L, 12, 8, 20000),
                                               (L, 40, 3, 20000), (8.0, 30, 4, 60000)])
def test_chains_stay_in_the_target_distribution(box, step, moves, P):
    # the small box has a = 0.25: every acceptance probability matters
    m = oracle.rbe_metropolis(11, step, P, box, ALPHA, moves)
    assert not np.any(np.all(m == 0, axis=1))
    r, p = exact_marginal(box)
    for d in range(3):
        counts = np.array([(m[:, d] == j).sum() for j in r])
        assert chi2_pvalue(counts, p * P) > 1e-3, (step, d)


def test_chains_move_and_freeze_without_moves():
    P = 2000
    m1 = oracle.rbe_metropolis(3, 5, P, L, ALPHA, 8)
    m2 = oracle.rbe_metropolis(3, 6, P, L, ALPHA, 8)
    moved = np.any(m1 != m2, axis=1).mean()
    assert moved > 0.5
    for d in range(3):  # every axis is proposed
        assert np.mean(m1[:, d] != m2[:, d]) > 0.2, d
    # each step changes a coordinate by at most `moves` in total
    assert np.abs(m2 - m1).sum(axis=1).max() <= 8
    m0 = oracle.rbe_sample(3, 0, P, L, ALPHA)
    assert np.array_equal(oracle.rbe_metropolis(3, 9, P, L, ALPHA, 0), m0)
    assert np.array_equal(oracle.rbe_metropolis(3, 0, P, L, ALPHA, 8), m0)


def test_acceptance_table_closed_form():
    A = oracle.metropolis_table(L, ALPHA)
    a = math.pi ** 2 / (ALPHA * L * L)
    for k in (0, 1, 5, 20):
        assert abs(float(A[k]) / 2.0 ** 64 - math.exp(-a * (2 * k + 1))) < 1e-15
    assert np.all(np.diff(A.astype(np.float64)) <= 0)
