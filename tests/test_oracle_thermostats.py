"""Pins of the oracle's Langevin and Nose-Hoover thermostats (Sec. 2.1).

With every force switched off (no charges, eps = 0) the thermostats act alone and
their discrete dynamics have closed forms:

  * Langevin: the half-step velocity follows x' = (1 - gamma dt) x + dt sqrt(2 gamma
    T0/dt) G, and the full-step velocity the oracle returns, a = x (1 - gamma dt/2)
    + dt/2 sqrt(2 gamma T0 / dt) G, has the stationary variance T0 exactly; the
    relaxation of <a^2> from T_init follows (1 - gamma dt)^(2n) to first order;
  * Nose-Hoover: dK/dt = -2 xi K, dxi/dt = (2K - g T0)/Q.  Small oscillations of K
    about g T0 / 2 have the angular frequency sqrt(2 g T0 / Q) = sqrt(2)/tau, and
    K + Q xi^2 / 2 + g T0 int xi dt is conserved.
The Box-Muller normals are checked against the standard normal distribution.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2407_09315_b300 import synth


def free_system(n, T0, seed):
    s = synth.electrolyte(n, seed=seed, T0=T0, dmin_factor=0.0)
    return s, np.zeros(n), np.zeros(1)


def run(s, q, eps, steps, thermostat, T0, tau, dt, xi=0.0, v=None, u=None, step0=0):
    F = np.zeros((s.n, 3))
    return oracle.vv(s.u if u is None else u, s.v if v is None else v, F, q, s.types, eps,
                     s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 8, seed=5, step0=step0, dt=dt,
                     n_steps=steps, thermostat=thermostat, T0=T0, tau=tau, xi=xi,
                     return_xi=True)


def test_langevin_normals_are_standard_normal():
    from scipy import stats

    g = np.array([oracle.langevin_normals(7, i, s) for i in range(2500) for s in (1, 2, 3, 4)])
    x = g.ravel()
    assert abs(x.mean()) < 4.0 / math.sqrt(len(x))
    assert abs(x.var() - 1.0) < 4.0 * math.sqrt(2.0 / len(x))
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the three components of one draw are uncorrelated (Box-Muller pairs)
    c = np.corrcoef(g.T)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        assert abs(c[a, b]) < 4.0 / math.sqrt(len(g)), (a, b, c[a, b])
    # and so are the squares (a cos/cos pair would correlate them)
    c2 = np.corrcoef((g * g).T)
    assert abs(c2[0, 1]) < 4.0 / math.sqrt(len(g))
    # different atoms, steps and replicas draw different numbers
    assert not np.allclose(oracle.langevin_normals(7, 1, 1), oracle.langevin_normals(7, 1, 2))
    assert not np.allclose(oracle.langevin_normals(7, 1, 1), oracle.langevin_normals(7, 2, 1))
    assert not np.allclose(oracle.langevin_normals(7, 1, 1, replica=1),
                           oracle.langevin_normals(7, 1, 1))


def test_langevin_stationary_temperature_is_T0():
    T0, tau, dt = 1.0, 0.05, 0.005  # gamma dt = 0.1
    s, q, eps = free_system(3000, 2.0, 11)
    u, v, F, _ = run(s, q, eps, 60, 2, T0, tau, dt)  # burn-in: (1 - gamma dt)^120 ~ 3e-6
    samples = []
    for k in range(12):
        s2 = s
        u, v, F2, _ = oracle.vv(u, v, F, q, s.types, eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 8,
                                seed=5, step0=60 + 20 * k, dt=dt, n_steps=20, thermostat=2,
                                T0=T0, tau=tau, return_xi=True)
        F = F2
        samples.append(np.mean(v * v))
    m = float(np.mean(samples))
    assert abs(m - T0) < 0.015 * T0, m


def test_langevin_relaxation_rate():
    # from T_init = 3, <a^2> - T0 decays by (1 - gamma dt)^2 per step to first order
    T0, tau, dt = 1.0, 0.2, 0.002  # gamma dt = 0.01
    s, q, eps = free_system(4000, 3.0, 12)
    v0 = np.mean(s.v * s.v)
    _, v, _, _ = run(s, q, eps, 40, 2, T0, tau, dt)
    pred = T0 + (v0 - T0) * (1 - dt / tau) ** 80
    assert abs(np.mean(v * v) - pred) < 0.03 * pred


def test_nose_hoover_oscillation_period_and_invariant():
    T0, tau, dt = 1.0, 0.1, 0.001
    s, q, eps = free_system(300, 1.05, 13)  # 5% above T0: small oscillation
    g = 3.0 * s.n - 3.0
    Q = g * T0 * tau * tau
    u, v, xi = s.u, s.v, 0.0
    K = [0.5 * np.sum(v * v)]
    H0 = K[0]
    eta = 0.0
    F = np.zeros((s.n, 3))
    Hs = []
    for k in range(600):
        xi_old = xi
        u, v, F, xi = oracle.vv(u, v, F, q, s.types, eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 8,
                                seed=5, step0=k, dt=dt, n_steps=1, thermostat=3, T0=T0, tau=tau,
                                xi=xi, return_xi=True)
        eta += 0.5 * (xi_old + xi) * dt
        K.append(0.5 * np.sum(v * v))
        Hs.append(K[-1] + 0.5 * Q * xi * xi + g * T0 * eta)
    K = np.array(K)
    # starting hot, xi grows and K falls first
    assert K[20] < K[0]
    # period from the crossings of the mean
    d = K - g * T0 / 2.0
    cross = np.where(np.sign(d[1:]) != np.sign(d[:-1]))[0]
    period = 2.0 * np.mean(np.diff(cross)) * dt
    assert abs(period - 2.0 * math.pi * tau / math.sqrt(2.0)) < 0.03 * period
    assert np.max(np.abs(np.array(Hs) - H0)) < 1e-4 * H0


def test_berendsen_is_unchanged_by_the_new_thermostats():
    s, q, eps = free_system(200, 2.0, 14)
    _, v1, _, xi = run(s, q, eps, 20, 1, 1.0, 0.1, 0.001)
    T = np.sum(v1 * v1) / (3.0 * s.n - 3.0)
    T_init = np.sum(s.v * s.v) / (3.0 * s.n - 3.0)
    assert abs(T - (1.0 + (1 - 0.01) ** 20 * (T_init - 1.0))) < 1e-10
    assert xi == 0.0
