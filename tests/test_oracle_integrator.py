"""Pins of the oracle's velocity-Verlet + Berendsen integrator (Sec. 2.1, Sec. 4).

  * with no forces the Berendsen rescale relaxes the temperature geometrically,
    T_n - T0 = (1 - dt/tau)^n (T_0 - T0) (closed form of lambda^2 = 1 + (dt/tau)(T0/T - 1));
  * with deterministic forces (no RBE, exact list) the kick-drift-kick scheme is
    time reversible: run n steps, flip the velocities, run n steps, and the
    fixed-point positions come back;
  * free flight: with no forces the positions drift by rint(v dt 2^32 / L) per
    step, wrapping modulo the box.
"""
import numpy as np

import oracle
from paper_2407_09315_b300 import synth

TWO32 = 2.0 ** 32


def _temperature(v):
    n = len(v)
    return np.sum(v * v) / (3.0 * n - 3.0)


def test_berendsen_relaxation_closed_form():
    s = synth.electrolyte(200, seed=1, T0=2.0)
    q = np.zeros(s.n)
    eps = np.zeros(1)
    dt, tau, T0 = 0.001, 0.1, 1.0
    F = np.zeros((s.n, 3))
    T_init = _temperature(s.v)
    u, v, F = oracle.vv(s.u, s.v, F, q, s.types, eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 10,
                        seed=0, step0=0, dt=dt, n_steps=20, thermostat=1, T0=T0, tau=tau)
    T20 = _temperature(v)
    ref = T0 + (1 - dt / tau) ** 20 * (T_init - T0)
    assert abs(T20 - ref) < 1e-10 * ref
    # free flight: positions advanced by the rounded displacement of each step
    c = dt * (TWO32 / s.L)
    assert np.all(np.abs(F) == 0)


def test_free_flight_drift_and_wrap():
    n = 4
    u = np.array([[0, 10, 2 ** 32 - 5], [7, 7, 7], [2 ** 31, 1, 2], [3, 4, 5]], dtype=np.uint32)
    v = np.array([[1.0, -2.0, 3.0], [0.0, 0.5, -0.5], [10.0, 0, 0], [-1, -1, -1]])
    L, dt = 10.0, 0.01
    u1, v1, _ = oracle.vv(u, v, np.zeros((n, 3)), np.zeros(n), np.zeros(n, np.int32),
                          np.zeros(1), np.ones(1), L, 0.62, 1.0, 1.0, 2.0, 4, 4, 0, 0, dt, 3,
                          thermostat=0)
    du = np.rint(v * (dt * TWO32 / L)).astype(np.int64)
    ref = (u.astype(np.int64) + 3 * du) % 2 ** 32
    assert np.array_equal(u1.astype(np.int64), ref)
    assert np.array_equal(v1, v)


def test_kick_drift_kick_is_time_reversible():
    s = synth.electrolyte(128, seed=3, n_types=2, T0=1.0)
    q = np.zeros(s.n)  # no charges: RBE vanishes, the list is exact -> deterministic forces
    kw = dict(q=q, types=s.types, eps=s.eps, sig=s.sig, L=s.L, alpha=0.62, coulomb_k=1.0,
              r_core=2.0, r_cut=3.5, p=10, P=4, seed=0, dt=0.002, thermostat=0, exact=True)
    F0, _ = oracle.forces(s.u, q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 4, 0, 0,
                          exact=True)
    u1, v1, F1 = oracle.vv(s.u, s.v, F0, step0=0, n_steps=25, **kw)
    moved = np.abs((u1.astype(np.int64) - s.u.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31)
    assert moved.max() > 1e5
    u2, v2, _ = oracle.vv(u1, -v1, F1, step0=25, n_steps=25, **kw)
    back = (u2.astype(np.int64) - s.u.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.max(np.abs(back)) <= 1
    assert np.allclose(-v2, s.v, rtol=1e-9, atol=1e-9)


def test_nve_energy_error_is_second_order_in_dt():
    # LJ fluid, exact lists, no charges: velocity Verlet's energy error over a
    # fixed time span falls by 4 when dt halves.
    s = synth.electrolyte(128, seed=5, n_types=1, T0=0.5)
    q = np.zeros(s.n)
    args = (s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 4)

    def energy(u, v):
        _, E = oracle.forces(u, q, *args, 0, 0, exact=True)
        return E[1] + 0.5 * np.sum(v * v)

    F0, _ = oracle.forces(s.u, q, *args, 0, 0, exact=True)
    E0 = energy(s.u, s.v)
    err = []
    for dt, n in ((0.002, 50), (0.001, 100), (0.0005, 200)):
        u, v, F = oracle.vv(s.u, s.v, F0, q, *args, seed=0, step0=0, dt=dt, n_steps=n,
                            thermostat=0, exact=True)
        err.append(abs(energy(u, v) - E0))
    assert 3.0 < err[0] / err[1] < 5.5
    assert 3.0 < err[1] / err[2] < 5.5
    assert err[2] < 1e-3 * 0.5 * np.sum(s.v * s.v)
