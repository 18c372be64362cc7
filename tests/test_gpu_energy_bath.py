"""Energy bath (thermostat 4, the NVE scheme of Sec. 2.1 in the reading the oracle
states) of rbmd_step against the oracle's integrator, and its invariants on the
GPU: tau = dt holds K + U at the bath energy, an infinite coupling time is the
plain step bit for bit, the bath energy is taken from the start state unless set,
and a checkpoint with the bath energy resumes bit-identically."""
import math

import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

ORC = (0.62, 1.0, 2.0, 3.5, 10)  # alpha, coulomb_k, r_core, r_cut, p (the test defaults)


def _wrap_diff(a, b):
    return (a.astype(np.int64) - b.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31


def _oracle_H(s, P, seed, step=0):
    """Forces, kinetic energy, potential and the sum of the magnitudes of the
    energy terms (the scale of the rounding of K + U) of the system's state."""
    F, E = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, *ORC, P, seed, step)
    K = 0.5 * float(np.sum(np.asarray(s.v, dtype=np.float64) ** 2))
    return F, K, float(np.sum(E)), K + float(np.sum(np.abs(E)))


def test_fp64_trajectory_matches_oracle():
    s = synth.electrolyte(600, seed=31, charges="2:1", n_types=2, T0=1.3)
    F0, K0, U0, _ = _oracle_H(s, 50, 4)
    E0 = K0 + U0 + 0.05 * K0  # a bath above the start energy: the rescale acts
    ctx, _ = make_ctx(s, rb.FP64, rbe_P=50, seed=4, dt=0.001, thermostat=4, tau_T=0.02)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.set_thermostat_state([E0])
    ctx.step(10)
    u, v, st = ctx.get_state_u()
    assert st == 10
    uo, vo, _, xo = oracle.vv(s.u, s.v, F0, s.q, s.types, s.eps, s.sig, s.L, *ORC, 50, seed=4,
                              step0=0, dt=0.001, n_steps=10, thermostat=4, tau=0.02, xi=E0,
                              return_xi=True)
    assert np.max(np.abs(_wrap_diff(to_np(u).astype(np.int64) % 2 ** 32, uo))) <= 2
    assert rel_err(to_np(v), vo) < 1e-9
    assert ctx.thermostat_state()[0] == E0 == xo
    # the bath acted: the plain step's velocities are elsewhere
    _, vn, _ = oracle.vv(s.u, s.v, F0, s.q, s.types, s.eps, s.sig, s.L, *ORC, 50, seed=4,
                         step0=0, dt=0.001, n_steps=10)
    assert rel_err(vn, vo) > 1e-4
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_bath_energy_is_taken_from_the_start_state(prec):
    s = synth.electrolyte(800, seed=32, charges="1:1", n_types=2)
    ctx, _ = make_ctx(s, prec, rbe_P=40, seed=6, dt=0.001, thermostat=4, tau_T=0.05)
    ctx.set_state_u(s.u, vel=s.v, step=3)
    assert math.isnan(ctx.thermostat_state()[0])
    ctx.step(1)
    _, K0, U0, scale = _oracle_H(s, 40, 6, step=3)
    tol = 1e-10 if prec == rb.FP64 else 1e-5
    assert abs(ctx.thermostat_state()[0] - (K0 + U0)) <= tol * scale
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_tau_dt_holds_the_total_energy_at_the_bath_energy(prec):
    s = synth.electrolyte(1500, seed=33, charges="2:1", n_types=2, T0=1.1)
    dt = 0.002
    ctx, _ = make_ctx(s, prec, rbe_P=60, seed=7, dt=dt, thermostat=4, tau_T=dt)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(1)
    E0 = ctx.thermostat_state()[0]
    tol = 1e-10 if prec == rb.FP64 else 1e-5
    for k in range(2, 6):
        ctx.step(1)
        e = ctx.energy(k)
        H = e["e_kinetic"] + e["e_potential"]
        assert abs(H - E0) <= tol * (abs(e["e_kinetic"]) + abs(e["e_potential"])), (k, H, E0)
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_infinite_coupling_time_is_the_plain_step(prec):
    # lambda = 1 exactly; the bath's steps run the energy variant of the pair
    # kernel, whose forces may differ from the plain kernel's in the last bit, so
    # the runs agree to rounding: velocities within the precision's tolerance and
    # positions within the drift's rounding (1 + 2 |dv| dt 2^32/L units a step)
    s = synth.electrolyte(1200, seed=34, charges="1:1", n_types=2)
    runs = []
    for thermostat, tau in ((4, 1e300), (0, 0.1)):
        ctx, _ = make_ctx(s, prec, rbe_P=40, seed=8, dt=0.002, thermostat=thermostat,
                          tau_T=tau)
        ctx.set_state_u(s.u, vel=s.v, step=0)
        ctx.step(2)
        ctx.step(3)  # the captured step graph replayed
        runs.append(ctx.get_state_u())
        ctx.close()
    (ua, va, _), (ub, vb, _) = runs
    va, vb = to_np(va), to_np(vb)
    assert rel_err(va, vb) < (1e-12 if prec == rb.FP64 else 1e-5)
    c = 0.002 * (4294967296.0 / s.L)
    allowed = 5 * (1.0 + 2.0 * float(np.abs(va - vb).max()) * c)
    du = _wrap_diff(to_np(ua).astype(np.int64) % 2 ** 32, to_np(ub).astype(np.int64) % 2 ** 32)
    assert np.max(np.abs(du)) <= allowed


def test_checkpoint_with_the_bath_energy_resumes_bit_identically():
    import torch

    s = synth.electrolyte(700, seed=35, charges="2:1", n_types=2, T0=1.4)
    kw = dict(rbe_P=40, seed=9, dt=0.001, thermostat=4, tau_T=0.03)
    a, _ = make_ctx(s, rb.FP64, **kw)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(6)
    ua, va, _ = a.get_state_u()
    b, _ = make_ctx(s, rb.FP64, **kw)
    b.set_state_u(s.u, vel=s.v, step=0)
    b.step(3)
    u3, v3, st = b.get_state_u()
    E0 = b.thermostat_state()
    c, _ = make_ctx(s, rb.FP64, **kw)
    c.set_state_u(u3, vel=v3, step=st)
    c.set_thermostat_state(E0)
    c.step(3)
    uc, vc, stc = c.get_state_u()
    assert stc == 6 and c.thermostat_state()[0] == E0[0]
    assert torch.equal(uc, ua) and torch.equal(vc, va)
    for x in (a, b, c):
        x.close()
