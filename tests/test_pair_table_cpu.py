"""The erfc-Coulomb look-up table (Sec. 3.3's look-up method), built by the library
on the host and checked here without a GPU against the closed forms evaluated with
Python's own math.erfc/math.exp:

  force factor  f(s) = [erfc(sqrt(alpha s))/sqrt(s) + 2 sqrt(alpha/pi) e^{-alpha s}] / s
  energy factor e(s) = erfc(sqrt(alpha s))/sqrt(s),   s = r^2,

with the bare terms s^{-3/2}, s^{-1/2} added back below the knot i0.
"""
import math

import numpy as np
import pytest

import paper_2407_09315_b300 as rb


def exact(alpha, s):
    r = math.sqrt(s)
    e = math.erfc(math.sqrt(alpha) * r) / r
    f = (e + 2.0 * math.sqrt(alpha / math.pi) * math.exp(-alpha * s)) / s
    return f, e


def interp(i0, inv_h, coef, s):
    n = coef.shape[0]
    u = s * inv_h
    k = min(int(u), n - 1)
    t = u - k
    cf, ce = coef[k, 0], coef[k, 1]
    f = ((cf[3] * t + cf[2]) * t + cf[1]) * t + cf[0]
    e = ((ce[3] * t + ce[2]) * t + ce[1]) * t + ce[0]
    if k < i0:
        f += s ** -1.5
        e += s ** -0.5
    return f, e


@pytest.mark.parametrize("alpha,r_cut,n,tol", [(0.62, 3.5, 1024, 2e-9), (0.62, 3.5, 8192, 2e-12),
                                               (0.362, 12.0, 8192, 1e-11), (1.5, 2.5, 4096, 5e-12)])
def test_table_matches_closed_forms(alpha, r_cut, n, tol):
    i0, inv_h, coef = rb.pair_table(alpha, r_cut, n)
    h = 1.0 / inv_h
    assert abs(h * n - r_cut ** 2 * (1 + 1e-6)) < 1e-12 * r_cut ** 2
    assert i0 == math.ceil((r_cut ** 2 / 9.0) / h)
    rng = np.random.default_rng(n)
    for s in rng.uniform((0.15 * r_cut) ** 2, r_cut ** 2, 4000):
        f, e = interp(i0, inv_h, coef, float(s))
        fx, ex = exact(alpha, float(s))
        assert abs(f - fx) <= tol * abs(fx), (s, f, fx)
        assert abs(e - ex) <= tol * abs(ex), (s, e, ex)


def test_table_is_continuous_and_reaches_zero_distance():
    alpha, r_cut, n = 0.62, 3.5, 2048
    i0, inv_h, coef = rb.pair_table(alpha, r_cut, n)
    for k in range(n - 1):
        for c in range(2):
            end = coef[k, c].sum()       # value at t = 1
            start = coef[k + 1, c, 0]   # value at t = 0 of the next piece
            if k + 1 == i0:  # remainder below the knot, full factor above
                s = (k + 1) / inv_h
                end += s ** (-1.5 if c == 0 else -0.5)
            assert abs(end - start) <= 1e-12 * max(1.0, abs(start))
    # the remainders at s = 0: f - s^{-3/2} -> -(4/3) alpha^{3/2}/sqrt(pi),
    # e - s^{-1/2} -> -2 sqrt(alpha/pi)
    assert abs(coef[0, 0, 0] + 4.0 / 3.0 * alpha ** 1.5 / math.sqrt(math.pi)) < 1e-12
    assert abs(coef[0, 1, 0] + 2.0 * math.sqrt(alpha / math.pi)) < 1e-12


def test_table_rejects_bad_arguments():
    for args in [(0.0, 3.5, 1024), (0.62, -1.0, 1024), (0.62, 3.5, 8)]:
        with pytest.raises(rb.RBMDError):
            rb.pair_table(*args)
