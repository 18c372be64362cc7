"""Pins of the oracle's random batch Ewald (Sec. 2.2, Eq. 12, Algorithm 1).

  * unbiasedness (stated below Eq. 12): the force averaged over many
    independent steps converges to the full Ewald Fourier force (Eq. 11),
    component z-scores ~ N(0, 1); likewise the energy estimate;
  * variance proportional to 1/P (stated below Eq. 12);
  * every mode kept with Gaussian weights reproduces Eq. 11 exactly;
  * the RBE force is minus the gradient of its energy estimate (fixed draws);
  * the RBE forces of one step sum to zero.
"""
import numpy as np
import pytest
from scipy import stats

import oracle

TWO32 = 2.0 ** 32


def _system(n, seed, dmin=0.8):
    from paper_2407_09315_b300 import synth
    return synth.electrolyte(n, seed=seed, charges="1:1", n_types=1, dmin_factor=dmin)


def test_rbe_unbiased_against_ewald():
    s = _system(32, 1)
    alpha, P, K = 0.62, 16, 3000
    M = oracle.sampler_M(s.L, alpha)
    ref = oracle.ewald(s.u, s.q, s.L, alpha, 1.0, 2.0, M)
    F = np.zeros((K, s.n, 3))
    E = np.zeros(K)
    for k in range(K):
        F[k], E[k], _, _ = oracle.rbe_forces(s.u, s.q, s.L, alpha, 1.0, P, seed=5, step=k)
    mean = F.mean(0)
    se = F.std(0, ddof=1) / np.sqrt(K)
    z = ((mean - ref["F_recip"]) / se).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert np.max(np.abs(z)) < 4.5
    zE = (E.mean() - ref["E_recip"]) / (E.std(ddof=1) / np.sqrt(K))
    assert abs(zE) < 4.5
    # the per-step estimates really are noisy (not the exact force)
    assert np.mean(np.abs(F[0] - ref["F_recip"])) > 1e-3 * np.mean(np.abs(ref["F_recip"]))


def test_rbe_variance_scales_as_one_over_P():
    s = _system(32, 2)
    alpha, K = 0.62, 600
    Ps = [8, 32, 128]
    var = []
    for P in Ps:
        F = np.array([oracle.rbe_forces(s.u, s.q, s.L, alpha, 1.0, P, seed=9, step=k)[0]
                      for k in range(K)])
        var.append(F.var(0, ddof=1).mean())
    slope = np.polyfit(np.log(Ps), np.log(var), 1)[0]
    assert abs(slope + 1.0) < 0.1, slope


def test_all_modes_with_gaussian_weights_is_ewald():
    s = _system(24, 3)
    alpha = 0.8
    M = oracle.sampler_M(s.L, alpha)
    m, w = oracle.full_modes(s.L, alpha, M)
    F, E, _ = oracle.mode_forces(s.u, s.q, s.L, 1.0, m, w)
    ref = oracle.ewald(s.u, s.q, s.L, alpha, 1.0, 2.0, M)
    assert np.allclose(F, ref["F_recip"], rtol=1e-12, atol=1e-14)
    assert abs(E - ref["E_recip"]) < 1e-12 * abs(E)


def test_rbe_force_is_gradient_of_estimate():
    s = _system(16, 4)
    alpha, P, step = 0.62, 64, 17
    F, E, m, _ = oracle.rbe_forces(s.u, s.q, s.L, alpha, 1.0, P, seed=3, step=step)
    S = oracle.rbe_S(s.L, alpha)
    W = np.full(P, S / P)
    du = int(round(1e-5 * TWO32 / s.L))
    hx = du * s.L / TWO32
    for i in (0, 9):
        for d in range(3):
            up = s.u.copy(); dn = s.u.copy()
            up[i, d] = np.uint32((int(s.u[i, d]) + du) % 2 ** 32)
            dn[i, d] = np.uint32((int(s.u[i, d]) - du) % 2 ** 32)
            g = (oracle.mode_forces(up, s.q, s.L, 1.0, m, W)[1] -
                 oracle.mode_forces(dn, s.q, s.L, 1.0, m, W)[1]) / (2 * hx)
            assert abs(-g - F[i, d]) < 1e-6 * (abs(F[i, d]) + 1.0)


def test_rbe_forces_sum_to_zero_and_match_structure_factor():
    s = _system(200, 5)
    F, E, m, rho = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, 100, seed=0, step=2)
    assert np.linalg.norm(F.sum(0)) < 1e-11 * np.abs(F).sum()
    # rho(k) of Eq. 9 by a direct complex sum
    x = s.x
    k = 2 * np.pi * m / s.L
    rho_ref = (s.q[None, :] * np.exp(1j * (k @ x.T))).sum(1)
    assert np.allclose(rho, rho_ref, rtol=1e-11, atol=1e-11)
    # selected-atom evaluation equals the full one
    sel = np.array([3, 77, 150])
    Fs = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, 100, seed=0, step=2, sel=sel)[0]
    assert np.array_equal(Fs, F[sel])
