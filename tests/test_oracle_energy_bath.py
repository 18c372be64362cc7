"""Pins of the oracle's energy bath (thermostat 4, the NVE scheme of Sec. 2.1).

The paper names an energy-stable scheme with an energy bath for NVE runs but does
not state its steps; the oracle's reading is a Berendsen-type relaxation of the
total energy H = K + U toward the bath energy E0:

    K -> K + (dt/tau)(E0 - U - K)   (velocities scaled by lambda = sqrt of the ratio)

with U the potential energy of the new configuration (the step's random batches)
and lambda clamped to [0.8, 1.25].  The pins follow from that definition alone:

  * tau = dt: after every step K + U = E0, with U evaluated independently;
  * tau -> infinity: lambda = 1 exactly, the plain velocity-Verlet trajectory;
  * no forces (U = 0): K_n - E0 = (1 - dt/tau)^n (K_0 - E0) in closed form, and the
    scheme is the Berendsen thermostat with target temperature 2 E0 / g;
  * the clamp: lambda^2 = 1.5625 or 0.64 exactly when the bath is far away.
"""
import numpy as np

import oracle
from paper_2407_09315_b300 import synth

ARGS = dict(alpha=0.62, coulomb_k=1.0, r_core=2.0, r_cut=3.5, p=10, P=30)


def _forces(s, q, eps, step):
    return oracle.forces(s.u, q, s.types, eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                         ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["P"], 9, step)


def _vv(s, u, v, F, q, eps, step0, n_steps, thermostat, tau, xi, dt=0.002, T0=1.0):
    return oracle.vv(u, v, F, q, s.types, eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                     ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["P"], seed=9, step0=step0,
                     dt=dt, n_steps=n_steps, thermostat=thermostat, T0=T0, tau=tau, xi=xi,
                     return_xi=True)


def _kinetic(v):
    return 0.5 * float(np.sum(np.asarray(v) ** 2))


def _potential(s, u, q, eps, step):
    _, E = oracle.forces(u, q, s.types, eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                         ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["P"], 9, step)
    return float(np.sum(E))


def test_tau_equal_dt_puts_the_total_energy_at_the_bath_energy():
    s = synth.electrolyte(300, seed=41, charges="2:1", n_types=2, T0=1.2)
    F, E = _forces(s, s.q, s.eps, 0)
    H0 = _kinetic(s.v) + float(np.sum(E))
    u, v = s.u, s.v
    for E0 in (H0, H0 + 0.1 * _kinetic(s.v)):
        u, v, Fk = s.u, s.v, F
        for k in range(4):
            u, v, Fk, xo = _vv(s, u, v, Fk, s.q, s.eps, k, 1, 4, 0.002, E0)
            assert xo == E0  # the bath energy is state, not changed by a step
            U = _potential(s, u, s.q, s.eps, k + 1)
            K = _kinetic(v)
            assert abs(K + U - E0) <= 1e-11 * (abs(K) + abs(U)), (k, K + U - E0)


def test_infinite_coupling_time_is_plain_velocity_verlet():
    s = synth.electrolyte(300, seed=42, charges="1:1", n_types=1)
    F, E = _forces(s, s.q, s.eps, 0)
    E0 = _kinetic(s.v) + float(np.sum(E)) + 5.0
    ub, vb, Fb, _ = _vv(s, s.u, s.v, F, s.q, s.eps, 0, 3, 4, 1e300, E0)
    un, vn, Fn, _ = _vv(s, s.u, s.v, F, s.q, s.eps, 0, 3, 0, 0.1, 0.0)
    assert np.array_equal(ub, un) and np.array_equal(vb, vn) and np.array_equal(Fb, Fn)


def test_without_forces_the_kinetic_energy_relaxes_geometrically_like_berendsen():
    n = 400
    s = synth.electrolyte(n, seed=43, T0=1.0, dmin_factor=0.0)
    q0, eps0 = np.zeros(n), np.zeros(1)
    assert _potential(s, s.u, q0, eps0, 0) == 0.0
    dt, tau = 0.002, 0.02  # dt / tau = 0.1
    K0 = _kinetic(s.v)
    E0 = 1.3 * K0
    u, v, F = s.u, s.v, np.zeros((n, 3))
    for k in range(1, 13):
        u, v, F, _ = _vv(s, u, v, F, q0, eps0, k - 1, 1, 4, tau, E0, dt=dt)
        want = E0 + (1.0 - dt / tau) ** k * (K0 - E0)
        assert abs(_kinetic(v) - want) <= 1e-12 * E0, (k, _kinetic(v), want)
    # the same run under Berendsen with T0 = 2 E0 / g
    g = 3.0 * n - 3.0
    ub, vb, _, _ = _vv(s, s.u, s.v, np.zeros((n, 3)), q0, eps0, 0, 12, 1, tau, 0.0, dt=dt,
                       T0=2.0 * E0 / g)
    vbath = _vv(s, s.u, s.v, np.zeros((n, 3)), q0, eps0, 0, 12, 4, tau, E0, dt=dt)[1]
    assert np.max(np.abs(vb - vbath)) <= 1e-13 * np.max(np.abs(vb))


def test_far_bath_is_clamped():
    n = 200
    s = synth.electrolyte(n, seed=44, T0=1.0, dmin_factor=0.0)
    q0, eps0 = np.zeros(n), np.zeros(1)
    K0 = _kinetic(s.v)
    F = np.zeros((n, 3))
    for E0, lam2 in ((10.0 * K0, 1.5625), (-K0, 0.64), (0.0, 0.64)):
        _, v, _, _ = _vv(s, s.u, s.v, F, q0, eps0, 0, 1, 4, 0.0002, E0, dt=0.002)
        assert abs(_kinetic(v) - lam2 * K0) <= 1e-13 * K0, (E0, _kinetic(v) / K0)
    # at rest there is nothing to scale
    _, v, _, _ = _vv(s, s.u, np.zeros((n, 3)), F, q0, eps0, 0, 1, 4, 0.002, K0, dt=0.002)
    assert not np.any(v)
