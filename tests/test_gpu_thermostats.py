"""Langevin (2) and Nose-Hoover (3) thermostats of rbmd_step against the oracle's
integrator (same seeds, same Philox normals), and the Nose-Hoover checkpoint."""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu


def _wrap_diff(a, b):
    return (a.astype(np.int64) - b.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31


@pytest.mark.parametrize("thermostat", [2, 3])
def test_fp64_trajectory_matches_oracle(thermostat):
    s = synth.electrolyte(600, seed=23, charges="1:1", n_types=2, T0=1.3)
    ctx, _ = make_ctx(s, rb.FP64, rbe_P=50, seed=4, dt=0.001, thermostat=thermostat,
                      temperature=1.0, tau_T=0.05)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(10)
    u, v, st = ctx.get_state_u()
    assert st == 10
    u = to_np(u).astype(np.int64) % 2 ** 32
    F0, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 50, 4, 0)
    uo, vo, _, xo = oracle.vv(s.u, s.v, F0, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5,
                              10, 50, seed=4, step0=0, dt=0.001, n_steps=10,
                              thermostat=thermostat, T0=1.0, tau=0.05, return_xi=True)
    assert np.max(np.abs(_wrap_diff(u, uo))) <= 2
    assert rel_err(to_np(v), vo) < 1e-9
    if thermostat == 3:
        xi = ctx.thermostat_state()
        assert xi.shape == (1,) and abs(xi[0] - xo) <= 1e-9 * abs(xo) + 1e-12
    ctx.close()


@pytest.mark.parametrize("thermostat", [2, 3])
def test_fp32_steps_stay_close_to_oracle(thermostat):
    # FP32 steps one at a time against the oracle's own trajectory from the same
    # start (the oracle carries its force, Langevin force and Nose-Hoover variable
    # from step to step).  A step's drift adds rint(v dt 2^32/L) to u, so the
    # positions can drift apart by at most 1 + 2 |dv| dt 2^32/L units per step,
    # |dv| the largest velocity difference seen so far (FP32 Langevin noise is
    # built from 24-bit uniforms, so |dv| is larger there than rounding alone);
    # the velocities stay within the FP32 tolerance.
    s = synth.electrolyte(1000, seed=24, charges="1:1", n_types=1)
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=50, seed=3, dt=0.001, thermostat=thermostat, tau_T=0.1)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    uo, vo, xo = s.u, s.v, 0.0
    Fo, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 50, 3, 0)
    c = 0.001 * (4294967296.0 / s.L)
    allowed = 0.0
    dv = 0.0
    for k in range(3):
        ctx.step(1)
        uo, vo, Fo, xo = oracle.vv(uo, vo, Fo, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0,
                                   3.5, 10, 50, seed=3, step0=k, dt=0.001, n_steps=1,
                                   thermostat=thermostat, tau=0.1, xi=xo, return_xi=True)
        u, v, st = ctx.get_state_u()
        assert st == k + 1
        dv = max(dv, float(np.abs(to_np(v) - vo).max()))
        allowed += 1.0 + 2.0 * dv * c
        du = _wrap_diff(to_np(u).astype(np.int64) % 2 ** 32, uo)
        assert np.max(np.abs(du)) <= allowed, (k, np.max(np.abs(du)), allowed)
        assert rel_err(to_np(v), vo) < 1e-5, k
        if thermostat == 3:
            assert abs(ctx.thermostat_state()[0] - xo) <= 1e-5 * abs(xo) + 1e-9
    ctx.close()


def test_nose_hoover_checkpoint_resume():
    s = synth.electrolyte(800, seed=25, charges="2:1", n_types=2, T0=1.5)
    kw = dict(rbe_P=40, seed=6, dt=0.001, thermostat=3, temperature=1.0, tau_T=0.05)
    a, _ = make_ctx(s, rb.FP64, **kw)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(6)
    ua, va, _ = a.get_state_u()
    b, _ = make_ctx(s, rb.FP64, **kw)
    b.set_state_u(s.u, vel=s.v, step=0)
    b.step(3)
    u3, v3, st = b.get_state_u()
    xi3 = b.thermostat_state()
    assert abs(xi3[0]) > 0
    c, _ = make_ctx(s, rb.FP64, **kw)
    c.set_state_u(u3, vel=v3, step=st)
    c.set_thermostat_state(xi3)
    c.step(3)
    uc, vc, stc = c.get_state_u()
    assert stc == 6
    assert np.max(np.abs(_wrap_diff(to_np(uc), to_np(ua)))) <= 1
    assert rel_err(to_np(vc), to_np(va)) < 1e-10
    for x in (a, b, c):
        x.close()


def test_langevin_holds_the_target_temperature():
    # strong coupling, many steps: the instantaneous temperature settles at T0
    s = synth.electrolyte(4000, seed=26, charges="1:1", n_types=1, T0=2.0)
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=20, seed=8, dt=0.002, thermostat=2, temperature=1.0,
                      tau_T=0.02)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    Ts = []
    for _ in range(6):
        ctx.step(50)
        Ts.append(ctx.energy(0)["temperature"])
    assert abs(np.mean(Ts[2:]) - 1.0) < 0.05, Ts
    ctx.close()
