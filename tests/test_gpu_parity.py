"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Every case feeds both sides the same seeded synthetic electrolyte (exact
fixed-point positions) and the same (seed, step): the random modes and batches
are drawn independently on each side from the same Philox definition, so they
must agree exactly; forces and energies must agree within the stated tolerance.
Sizes span several tiles with a ragged tail (1000, 1537 and 4099 atoms).
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

PRECS = [rb.FP64, rb.FP32]


@pytest.fixture(scope="module")
def sys1000():
    return synth.config1()


@pytest.fixture(scope="module")
def sys_ragged():
    return synth.electrolyte(1537, seed=11, charges="2:1", n_types=3)


@pytest.fixture(scope="module")
def sys_4099():
    return synth.electrolyte(4099, seed=12, charges="2:1", n_types=4)


# ------------------------------------------------------------------ RBE
@pytest.mark.parametrize("prec", PRECS)
def test_modes_bit_exact(sys1000, prec):
    ctx, prm = make_ctx(sys1000, prec, rbe_P=100, seed=0)
    for step in (0, 1, 77, 123456):
        m, rho = ctx.rbe_modes(step)
        mo = oracle.rbe_sample(0, step, 100, sys1000.L, 0.62)
        assert np.array_equal(m, mo), step
    ctx.close()


def test_modes_bit_exact_large_box_and_replica():
    L = 170.99759466766966
    s = synth.electrolyte(2000, L=L, seed=5, dmin_factor=0.0)
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=200, seed=0xDEADBEEF12345, replica=3)
    for step in (0, 9):
        m, _ = ctx.rbe_modes(step)
        mo = oracle.rbe_sample(0xDEADBEEF12345, step, 200, L, 0.62, replica=3)
        assert np.array_equal(m, mo)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["sys1000", "sys_ragged", "sys_4099"])
def test_structure_factors(which, prec, request):
    s = request.getfixturevalue(which)
    ctx, _ = make_ctx(s, prec, rbe_P=200, seed=4)
    m, rho = ctx.rbe_modes(3)
    rho_o = oracle.structure_factor(s.u, s.q, s.L, m)
    scale = np.sqrt(np.sum(s.q ** 2))
    err = np.max(np.abs(rho - rho_o)) / scale
    assert err < (1e-12 if prec == rb.FP64 else 2e-6), err
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["sys1000", "sys_ragged", "sys_4099"])
def test_rbe_forces(which, prec, request):
    s = request.getfixturevalue(which)
    ctx, prm = make_ctx(s, prec, rbe_P=200, seed=4)
    for step in (0, 5):
        F = to_np(ctx.rbe_forces(step))
        Fo, Eo, _, _ = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, 200, seed=4, step=step)
        assert rel_err(F, Fo) < TOL[prec], (step, rel_err(F, Fo))
    # accumulate mode adds onto the output
    base = ctx.rbe_forces(0)
    twice = ctx.rbe_forces(0, out=base.clone(), accumulate=True)
    assert rel_err(to_np(twice), 2 * to_np(base)) < 1e-6
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_full_ewald_modes_reproduce_eq11(sys1000, prec):
    s = sys1000
    ctx, _ = make_ctx(s, prec, flags=rb.FULL_EWALD_MODES)
    F = to_np(ctx.rbe_forces(0))
    M = oracle.sampler_M(s.L, 0.62)
    e = oracle.ewald(s.u, s.q, s.L, 0.62, 1.0, 3.5, M)
    assert rel_err(F, e["F_recip"]) < TOL[prec]
    E = ctx.energy(0)
    assert abs(E["e_rbe"] - e["E_recip"]) < (1e-10 if prec == rb.FP64 else 1e-5) * abs(e["E_recip"])
    assert abs(E["e_self"] - e["E_self"]) < 1e-12 * abs(e["E_self"])
    ctx.close()


# ------------------------------------------------------------------ RBL
@pytest.mark.parametrize("cell_div", [1, 2])
@pytest.mark.parametrize("p", [10, 30])
@pytest.mark.parametrize("which", ["sys1000", "sys_ragged"])
def test_rbl_lists_bit_exact(which, p, cell_div, request):
    s = request.getfixturevalue(which)
    ctx, _ = make_ctx(s, rb.FP32, rbl_p=p, seed=9, cell_div=cell_div)
    for step in (0, 3):
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, p, 9, step)
        assert np.array_equal(nc, o["n_core"])
        assert np.array_equal(ns, o["n_shell"])
        assert np.array_equal(b, o["batch"])
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["sys1000", "sys_ragged", "sys_4099"])
def test_rbl_forces(which, prec, request):
    s = request.getfixturevalue(which)
    ctx, _ = make_ctx(s, prec, seed=2)
    for step in (0, 7):
        F = to_np(ctx.rbl_forces(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 2, step)
        Fo = o["F"] - o["Fsum"] / s.n
        assert rel_err(F, Fo) < TOL[prec], (step, rel_err(F, Fo))
        assert np.linalg.norm(F.sum(0)) < 1e-6 * np.abs(F).sum()
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_rbl_exact_mode(sys_ragged, prec):
    s = sys_ragged
    ctx, _ = make_ctx(s, prec, flags=rb.RBL_EXACT)
    F = to_np(ctx.rbl_forces(0))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 0, 0, exact=True)
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[prec]
    ctx.close()


# ------------------------------------------------------------------ total + energies
@pytest.mark.parametrize("prec", PRECS)
def test_total_forces_and_energies(sys_4099, prec):
    s = sys_4099
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=6)
    F = to_np(ctx.forces(2))
    Fo, Eo = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 100, 6, 2)
    assert rel_err(F, Fo) < TOL[prec]
    E = ctx.energy(2)
    tol = 1e-10 if prec == rb.FP64 else 1e-5
    for k, ref in zip(("e_coul_real", "e_lj", "e_rbe", "e_self"), Eo):
        assert abs(E[k] - ref) <= tol * abs(ref) + 1e-12, (k, E[k], ref)
    assert abs(E["S"] - oracle.rbe_S(s.L, 0.62)) < 1e-12 * E["S"]
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 6, 2)
    assert E["max_shell"] == int(o["n_shell"].max())
    assert np.allclose(E["fsum_short"], o["Fsum"], rtol=1e-6, atol=1e-6 * np.abs(o["F"]).sum())
    ctx.close()


# ------------------------------------------------------------------ integrator
@pytest.mark.parametrize("thermostat", [0, 1])
def test_fp64_trajectory_matches_oracle(thermostat):
    s = synth.electrolyte(600, seed=13, charges="1:1", n_types=2, T0=1.0)
    ctx, _ = make_ctx(s, rb.FP64, rbe_P=50, seed=3, dt=0.001, thermostat=thermostat,
                      temperature=1.5, tau_T=0.1)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(10)
    u, v, st = ctx.get_state_u()
    assert st == 10
    u = to_np(u).astype(np.int64) % 2 ** 32
    F0, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 50, 3, 0)
    uo, vo, _ = oracle.vv(s.u, s.v, F0, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10,
                          50, seed=3, step0=0, dt=0.001, n_steps=10, thermostat=thermostat,
                          T0=1.5, tau=0.1)
    du = (u - uo.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.max(np.abs(du)) <= 2
    assert rel_err(to_np(v), vo) < 1e-9
    ctx.close()


def _wrap_diff(a, b):
    a = np.asarray(a).astype(np.int64)
    b = np.asarray(b).astype(np.int64)
    return (a - b + 2 ** 31) % 2 ** 32 - 2 ** 31


def _half_gap(y):
    """Distance of y from the nearest half-integer (where rint changes)."""
    return np.abs(np.abs(y - np.floor(y)) - 0.5)


@pytest.mark.parametrize("L,dt,vscale", [(17.1, 0.001, 1.0), (17.1, 0.001, 1000.0),
                                          (170.99759466766966, 0.002, 30.0)])
def test_fp32_drift_fixed_point_exact(L, dt, vscale):
    # Sec. 2.1 drift of the fixed-point state in isolation: with every force
    # exactly zero on both sides the velocities stay
    # the stored FP32 values and each step adds rint(v dt 2^32/L) to u.  The FP32
    # path forms that product from two floats (v * (dhi + dlo)); it must give the
    # oracle's FP64 integer exactly, except within 1e-5 units of a half-integer,
    # where a rounding of the product may decide (counted, and rare).  vscale up
    # to 1000 makes |v dt 2^32/L| reach 2.5e8, far beyond the 24-bit mantissa of
    # one float, so a dropped low part of the factor fails.
    n = 2000
    rng = np.random.default_rng(41)
    u0 = rng.integers(0, 2 ** 32, size=(n, 3), dtype=np.uint64).astype(np.uint32)
    v = (rng.standard_normal((n, 3)) * vscale).astype(np.float32).astype(np.float64)
    s = synth.System(L=L, u=u0, q=np.zeros(n), types=np.zeros(n, np.int32),
                     eps=np.array([0.0]), sig=np.array([1.0]), v=v)
    # the library skips both force parts (its forces are then exactly zero); the
    # oracle computes them with q = 0 and eps = 0, which is exactly zero too
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=20, seed=1, dt=dt, thermostat=0, r_core=1.0, r_cut=2.0,
                      flags=rb.NO_RBE | rb.NO_RBL)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    u_ref = u0.copy()
    F0 = np.zeros((n, 3))
    near_total = 0
    for k in range(3):
        ctx.step(1)
        u, vg, st = ctx.get_state_u()
        assert st == k + 1
        assert np.array_equal(to_np(vg), v)  # zero force: velocities unchanged, bit for bit
        u_ref, vo, _ = oracle.vv(u_ref, v, F0, s.q, s.types, s.eps, s.sig, L, 0.62, 1.0, 1.0, 2.0,
                                 10, 20, seed=1, step0=k, dt=dt, n_steps=1)
        assert np.array_equal(vo, v)
        du = _wrap_diff(to_np(u).astype(np.int64) % 2 ** 32, u_ref)
        near = _half_gap(v * (dt * (4294967296.0 / L))) < 1e-5
        assert np.all(du[~near] == 0), (k, np.argwhere(du[~near] != 0)[:5])
        assert np.all(np.abs(du[near]) <= 1)
        near_total += int(near.sum())
        u_ref = (to_np(u).astype(np.int64) % 2 ** 32).astype(np.uint32)  # continue from the GPU state
    assert near_total <= 3  # probability ~2e-5 per coordinate
    ctx.close()


@pytest.mark.parametrize("thermostat", [0, 1])
def test_fp32_step_positions_track_oracle_each_step(thermostat):
    # One FP32 step at a time from the GPU's own state (u_k, v_k): the oracle
    # takes the same state and its FP64 force of step k and makes one
    # velocity-Verlet step (Sec. 2.1).  The half-kick velocities differ by the
    # FP32 force error times dt/2 (measured per coordinate from the library's
    # force of step k) and by the FP32 rounding of v + F dt/2, so the drift
    # integer rint(v_half dt 2^32/L) may differ by one unit only where the
    # oracle's v_half dt 2^32/L lies within that difference (times 2) of a
    # half-integer; everywhere else u must be identical.  Velocities after the
    # step within the FP32 tolerance.
    s = synth.electrolyte(1000, seed=14, charges="1:1", n_types=1)
    dt = 0.001
    c = dt * (4294967296.0 / s.L)
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=50, seed=3, dt=dt, thermostat=thermostat)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    flips = 0
    for k in range(4):
        uk, vk, st = ctx.get_state_u()
        assert st == k
        uk = (to_np(uk).astype(np.int64) % 2 ** 32).astype(np.uint32)
        vk = to_np(vk)
        Fk, _ = oracle.forces(uk, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 50, 3, k)
        uo, vo, _ = oracle.vv(uk, vk, Fk, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10,
                              50, seed=3, step0=k, dt=dt, n_steps=1, thermostat=thermostat)
        Fg = to_np(ctx.forces(k))  # the force the step's first half kick uses
        ctx.step(1)
        u, v, _ = ctx.get_state_u()
        du = _wrap_diff(to_np(u).astype(np.int64) % 2 ** 32, uo)
        assert np.max(np.abs(du)) <= 1, k
        vh = vk + 0.5 * dt * Fk
        gap = _half_gap(vh * c)
        reach = c * (0.5 * dt * np.abs(Fg - Fk) + 2.0 ** -23 * (np.abs(vh) + 0.5 * dt * np.abs(Fk)))
        # a flipped coordinate sits within the velocity difference's reach of a tie
        bad = (du != 0) & (gap >= 2.0 * reach + 1e-6)
        assert not bad.any(), (k, gap[bad][:5], reach[bad][:5])
        flips += int(np.count_nonzero(du))
        assert rel_err(to_np(v), vo) < 1e-5, k
    assert flips <= 0.02 * 4 * 3 * s.n, flips
    ctx.close()


# ------------------------------------------------------------------ determinism, checkpoint
def test_bit_identical_runs_and_resume():
    import torch

    s = synth.electrolyte(3000, seed=15, charges="2:1", n_types=2)
    a, _ = make_ctx(s, rb.FP32, seed=1, thermostat=1)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(6)
    ua, va, _ = a.get_state_u()
    b, _ = make_ctx(s, rb.FP32, seed=1, thermostat=1)
    b.set_state_u(s.u, vel=s.v, step=0)
    b.step(3)
    u3, v3, st = b.get_state_u()
    c, _ = make_ctx(s, rb.FP32, seed=1, thermostat=1)
    c.set_state_u(u3, vel=v3, step=st)
    c.step(3)
    uc, vc, _ = c.get_state_u()
    b.step(3)
    ub, vb, _ = b.get_state_u()
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    # resume through a checkpoint: bit-identical to the unbroken run
    assert torch.equal(ua, uc) and torch.equal(va, vc)
    for x in (a, b, c):
        x.close()


def test_profiled_steps_match_unprofiled():
    import torch

    s = synth.electrolyte(2500, seed=16, charges="2:1", n_types=2)
    a, _ = make_ctx(s, rb.FP32, seed=1, thermostat=1)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(4)
    ua, va, _ = a.get_state_u()
    b, _ = make_ctx(s, rb.FP32, seed=1, thermostat=1)
    b.set_state_u(s.u, vel=s.v, step=0)
    b.profile(True)
    b.step(4)
    ub, vb, st = b.get_state_u()
    stages, n = b.profile_read(reset=True)
    assert st == 4 and n >= 3
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    for k in ("rbl_scan", "rbl_select", "rbl_force", "rho_partial", "rbe_force"):
        assert stages[k] > 0, k
    assert b.step_kernel_count() in (0, a.step_kernel_count())
    assert a.step_kernel_count() >= 10
    a.close()
    b.close()


@pytest.mark.parametrize("prec", PRECS)
def test_list_overflow_fallback_is_exact(sys_ragged, prec, monkeypatch):
    # Capacities far below the neighbour counts: (almost) every atom takes the
    # fused fallback path; lists, forces and energies must not change.
    s = sys_ragged
    monkeypatch.setenv("RBMD_LIST_CAPS", "3,7")
    ctx, _ = make_ctx(s, prec, seed=2, rbe_P=50)
    monkeypatch.delenv("RBMD_LIST_CAPS")
    nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(4))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 2, 4)
    assert np.array_equal(nc, o["n_core"]) and np.array_equal(ns, o["n_shell"])
    assert np.array_equal(b, o["batch"])
    F = to_np(ctx.rbl_forces(4))
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[prec]
    E = ctx.energy(4)
    assert abs(E["e_lj"] - o["E_lj"]) <= (1e-10 if prec == rb.FP64 else 1e-5) * abs(o["E_lj"])
    ctx.close()


@pytest.mark.parametrize("bits", [16, 8, 3])
@pytest.mark.parametrize("p", [10, 16, 30])
def test_truncated_selection_keys(sys_ragged, p, bits, monkeypatch):
    # the fast selection ranks packed keys (the priority's high word, its low bits
    # replaced by the member's list position) and hands an atom to the exact path
    # when two of its p + 1 smallest keys share their priority bits.  Keeping only
    # `bits` of them makes that common (3 bits: nearly every atom; 16: a few), and
    # the batches, their order (the FP32 pair sums follow it) and the oracle's
    # batches must not change.
    import torch

    s = sys_ragged
    ref, _ = make_ctx(s, rb.FP32, rbl_p=p, seed=12)
    monkeypatch.setenv("RBMD_SELECT_KEY_BITS", str(bits))
    ctx, _ = make_ctx(s, rb.FP32, rbl_p=p, seed=12)
    monkeypatch.delenv("RBMD_SELECT_KEY_BITS")
    for step in (0, 3):
        b = to_np(ctx.rbl_lists(step)[2]).astype(np.int64)
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, p, 12, step)
        assert np.array_equal(b, o["batch"]), step
        assert torch.equal(ctx.rbl_forces(step), ref.rbl_forces(step)), step
    ctx.close()
    ref.close()


@pytest.mark.parametrize("p", [10, 16, 30])
def test_exact_selection_path(sys_ragged, p, monkeypatch):
    # the exact slow path of the batch selection (taken by atoms whose priority
    # words tie) gives the same batches as the oracle when every atom takes it
    s = sys_ragged
    monkeypatch.setenv("RBMD_SELECT_EXACT", "1")
    ctx, _ = make_ctx(s, rb.FP32, rbl_p=p, seed=12)
    monkeypatch.delenv("RBMD_SELECT_EXACT")
    for step in (0, 2):
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, p, 12, step)
        assert np.array_equal(b, o["batch"]), step
    F = to_np(ctx.rbl_forces(2))
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[rb.FP32]
    ctx.close()
