"""The integrator's neighbour candidate lists (rbmd_step with a skin).

The step keeps, per atom, the atoms within r_cut + skin at the last rebuild and
classifies them exactly on the integer positions every step; a rebuild runs on
the device when an atom has moved more than skin/2 (or the sorted layout was
changed by another call).  The core list, N_s and the batch (Algorithm 2 step 1)
are then the sets of the per-step cell walk, and the forces are summed in an
order that does not depend on when rebuilds happen:

  * FP64 trajectories with and without the lists agree to rounding, for a skin
    that rebuilds almost every step and for the default one;
  * an FP32 run whose rebuilds are forced at other steps (other calls between
    the steps) is bit-identical to an unbroken run;
  * atoms beyond the lists' capacities take the exact fallback;
  * batched replicas with their shared rebuild decision match stand-alone runs.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu


def _wrap_diff(a, b):
    a = np.asarray(a).astype(np.int64)
    b = np.asarray(b).astype(np.int64)
    return (a - b + 2 ** 31) % 2 ** 32 - 2 ** 31


def _run(s, prec, n_steps, **kw):
    ctx, _ = make_ctx(s, prec, rbe_P=40, seed=5, dt=0.002, thermostat=1, **kw)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(n_steps)
    u, v, st = ctx.get_state_u()
    reb = ctx.candidate_rebuilds()
    ctx.close()
    return to_np(u).astype(np.int64) % 2 ** 32, to_np(v), st, reb


@pytest.mark.parametrize("skin", [0.003, 0.4])
def test_candidate_lists_match_cell_walk_fp64(skin):
    s = synth.electrolyte(2000, seed=61, charges="2:1", n_types=2, T0=1.5)
    u0, v0, _, r0 = _run(s, rb.FP64, 8, skin=-1.0)
    u1, v1, st, r1 = _run(s, rb.FP64, 8, skin=skin)
    assert st == 8 and r0 == 0
    if skin < 0.01:
        assert r1 >= 5, r1  # a tiny skin rebuilds nearly every step
    else:
        assert 1 <= r1 <= 2, r1  # the first step builds; 8 steps stay within 0.2
    assert np.max(np.abs(_wrap_diff(u1, u0))) <= 1
    assert rel_err(v1, v0) < 1e-12


@pytest.mark.parametrize("shape", ["el001", "lj001"])
def test_candidate_lists_p30_paper_shapes_fp64(shape):
    """Batches of p = 30 (the selection with 33 kept keys) in the paper's density-0.01
    regimes: the primitive electrolyte (r 6/12, about 63 shell members) and the LJ
    fluid (r 2.5/5, mostly whole shells): the trajectory through the candidate lists
    equals the cell walk's to rounding, and the oracle's."""
    if shape == "el001":
        s = synth.electrolyte(1500, seed=66, charges="1:1", n_types=1, density=0.01)
        kw = dict(alpha=0.362, r_core=6.0, r_cut=12.0, rbl_p=30, rbe_P=40, coulomb_k=3.5)
    else:
        s = synth.electrolyte(1500, seed=67, charges="1:1", n_types=1, density=0.01)
        s.q = s.q * 0.0
        kw = dict(alpha=0.62, r_core=2.5, r_cut=5.0, rbl_p=30, rbe_P=10, coulomb_k=1.0,
                  flags=rb.NO_RBE)
    out = []
    for skin in (-1.0, 0.4):
        ctx, _ = make_ctx(s, rb.FP64, seed=7, dt=0.002, thermostat=1, skin=skin, **kw)
        ctx.set_state_u(s.u, vel=s.v, step=0)
        F = to_np(ctx.forces(0))
        ctx.step(6)
        u, v, _ = ctx.get_state_u()
        out.append((F, to_np(u).astype(np.int64) % 2 ** 32, to_np(v), ctx.candidate_rebuilds()))
        ctx.close()
    (F0, u0, v0, r0), (F1, u1, v1, r1) = out
    assert r0 == 0 and r1 >= 1
    assert rel_err(F1, F0) < 1e-12
    assert np.max(np.abs(_wrap_diff(u1, u0))) <= 1
    assert rel_err(v1, v0) < 1e-12
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, kw["alpha"], kw["coulomb_k"], kw["r_core"],
                   kw["r_cut"], 30, 7, 0)
    if shape == "lj001":
        assert rel_err(F1, o["F"] - o["Fsum"] / s.n) < 1e-10


def test_fp64_candidate_trajectory_matches_oracle():
    s = synth.electrolyte(700, seed=62, charges="1:1", n_types=2, T0=1.2)
    ctx, _ = make_ctx(s, rb.FP64, rbe_P=30, seed=6, dt=0.002, thermostat=1, skin=0.01)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(6)
    u, v, _ = ctx.get_state_u()
    assert ctx.candidate_rebuilds() >= 2
    F0, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 30, 6, 0)
    uo, vo, _ = oracle.vv(s.u, s.v, F0, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10,
                          30, seed=6, step0=0, dt=0.002, n_steps=6, thermostat=1)
    assert np.max(np.abs(_wrap_diff(to_np(u).astype(np.int64) % 2 ** 32, uo))) <= 2
    assert rel_err(to_np(v), vo) < 1e-9
    ctx.close()


def test_rebuild_schedule_does_not_change_fp32_results():
    s = synth.electrolyte(3000, seed=63, charges="2:1", n_types=3)
    a, _ = make_ctx(s, rb.FP32, seed=2, thermostat=1)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(7)
    ua, va, _ = a.get_state_u()
    b, _ = make_ctx(s, rb.FP32, seed=2, thermostat=1)
    b.set_state_u(s.u, vel=s.v, step=0)
    for k in (2, 2, 3):
        b.step(k)
        b.rbl_lists(0)  # the cell walk re-sorts the atoms: the next step rebuilds
    ub, vb, st = b.get_state_u()
    assert st == 7
    assert b.candidate_rebuilds() > a.candidate_rebuilds()
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_candidate_overflow_takes_exact_fallback(prec, monkeypatch):
    s = synth.electrolyte(1500, seed=64, charges="2:1", n_types=2)
    ref, _ = make_ctx(s, prec, seed=3, skin=-1.0)
    monkeypatch.setenv("RBMD_LIST_CAPS", "4,12")
    ctx, _ = make_ctx(s, prec, seed=3)
    monkeypatch.delenv("RBMD_LIST_CAPS")
    for c in (ref, ctx):
        c.set_state_u(s.u, vel=s.v, step=0)
        c.step(3)
    u0, v0, _ = ref.get_state_u()
    u1, v1, _ = ctx.get_state_u()
    d = _wrap_diff(to_np(u1).astype(np.int64) % 2 ** 32, to_np(u0).astype(np.int64) % 2 ** 32)
    assert np.max(np.abs(d)) <= 1
    assert rel_err(to_np(v1), to_np(v0)) < (1e-12 if prec == rb.FP64 else 1e-5)
    ref.close()
    ctx.close()


def test_batch_candidates_match_standalone():
    sizes = [900, 2100, 1300]
    reps = [synth.electrolyte(n, seed=70 + r, charges="1:1", n_types=1) for r, n in enumerate(sizes)]
    dev = torch.device("cuda:0")
    cat = lambda k: np.concatenate([getattr(x, k) for x in reps])
    pos = torch.from_numpy(np.concatenate([x.x for x in reps])).to(dev, torch.float32)
    q = torch.from_numpy(cat("q")).to(dev, torch.float32)
    vel = torch.from_numpy(cat("v")).to(dev, torch.float32)
    ctx = rb.RBMD(pos, q, reps[0].eps, reps[0].sig, box_length=[x.L for x in reps],
                  n_atoms=sizes, seed=[3, 4, 5], replica=[0, 1, 2], precision=rb.FP32,
                  rbe_P=50, vel=vel, thermostat=1, skin=0.02, dt=0.002)
    ctx.set_state_u(cat("u"), vel=cat("v"), step=0)
    ctx.step(5)
    ub, vb, _ = ctx.get_state_u()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for r, x in enumerate(reps):
        c, _ = make_ctx(x, rb.FP32, rbe_P=50, seed=3 + r, replica=r, thermostat=1, skin=0.02,
                        dt=0.002)
        c.set_state_u(x.u, vel=x.v, step=0)
        c.step(5)
        u, v, _ = c.get_state_u()
        assert torch.equal(u, ub[off[r]:off[r + 1]]) and torch.equal(v, vb[off[r]:off[r + 1]])
        c.close()
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_force_calls_use_the_candidates(prec):
    """rbmd_forces and rbmd_forces_host evaluate through the candidate lists (rebuilt
    on the device only when an atom has moved more than skin/2): the forces equal
    the cell walk's (a context with skin < 0) to rounding, for a sequence of slightly
    moved states, and the rebuilds stay rare."""
    s = synth.electrolyte(3000, seed=65, charges="2:1", n_types=3)
    ctx, _ = make_ctx(s, prec, seed=5)
    ref, _ = make_ctx(s, prec, seed=5, skin=-1.0)
    tol = 1e-12 if prec == rb.FP64 else 2e-6
    rng = np.random.default_rng(5)
    u = s.u.astype(np.int64)
    scale = 2.0 ** 32 / s.L
    r0 = ctx.candidate_rebuilds()
    for k in range(6):
        # every atom moves up to 0.03 sigma per call: a rebuild about every fourth call
        u = (u + np.rint(rng.uniform(-0.03, 0.03, size=u.shape) * scale).astype(np.int64)) % 2 ** 32
        uu = u.astype(np.uint32)
        if k % 2 == 0:
            ctx.set_state_u(uu, step=k)
            F1 = to_np(ctx.forces(k))
        else:
            x = torch.from_numpy(uu.astype(np.float64) * (s.L / 2.0 ** 32))
            F1 = to_np(ctx.forces_host(x.to(ctx.dtype).pin_memory(), step=k))
        ref.set_state_u(ctx.get_state_u()[0], step=k)  # the state ctx encoded
        F0 = to_np(ref.forces(k))
        assert rel_err(F1, F0) < tol, (k, rel_err(F1, F0))
    assert ctx.candidate_rebuilds() - r0 <= 6
    ctx.close()
    ref.close()



@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_conditional_rebuild_node_matches_plain_graph_nodes(prec, monkeypatch):
    # the step graph puts the rebuild kernels in the body of a conditional node;
    # with RBMD_GRAPH_COND=0 they are plain graph nodes that return at once on
    # steps without a rebuild.  Same kernels, same bits; the node adds one kernel
    # (the one that opens it) and the body holds the nine rebuild kernels.
    s = synth.electrolyte(2500, seed=66, charges="2:1", n_types=2)
    runs = []
    for cond in ("1", "0"):
        monkeypatch.setenv("RBMD_GRAPH_COND", cond)
        ctx, _ = make_ctx(s, prec, seed=4, thermostat=1, dt=0.005, skin=0.02)  # rebuilds often
        ctx.set_state_u(s.u, vel=s.v, step=0)
        ctx.step(3)
        ctx.step(5)  # the captured graph replayed
        u, v, st = ctx.get_state_u()
        runs.append((u, v, ctx.step_kernel_count(), ctx.rebuild_kernel_count(),
                     ctx.candidate_rebuilds()))
        ctx.close()
    (ua, va, ka, ra, na), (ub, vb, kb, rb0, nb) = runs
    assert na == nb and na >= 3
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    assert rb0 == 0 and ra == 9
    assert ka + ra == kb + 1


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_calls_after_a_step_reuse_its_lists(prec):
    # force, energy and gradient calls right after a step skip the candidate check
    # (the step's check ran on these positions); a fresh context set to the same
    # state checks and rebuilds: the same lists, so the same forces bit for bit (each
    # atom's sum runs in a canonical order) and the same energies and gradients up to
    # the order of the sums over atoms, which follows the sorted layout
    s = synth.electrolyte(3000, seed=67, charges="2:1", n_types=2)
    a, _ = make_ctx(s, prec, seed=5, thermostat=1, dt=0.004)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(4)
    ua, va, st = a.get_state_u()
    b, _ = make_ctx(s, prec, seed=5, thermostat=1, dt=0.004)
    b.set_state_u(ua, vel=va, step=st)
    (Ea, Fa, Ga), (Eb, Fb, Gb) = ((c.energy(st), c.forces(st), c.energy_backward(st))
                                  for c in (a, b))
    tol = 1e-12 if prec == rb.FP64 else 2e-6
    assert Ea["max_shell"] == Eb["max_shell"]
    for k in ("e_coul_real", "e_lj", "e_rbe"):
        assert abs(Ea[k] - Eb[k]) <= tol * abs(Eb[k]), k
    assert np.allclose(Ea["virial"], Eb["virial"], rtol=tol, atol=tol * np.abs(Eb["virial"]).max())
    assert torch.equal(Fa, Fb)
    for x, y in zip(Ga, Gb):
        x, y = (to_np(x), to_np(y)) if isinstance(x, torch.Tensor) else (np.asarray(x), np.asarray(y))
        assert rel_err(x, y) <= tol
    a.close()
    b.close()


def test_a_step_after_a_cell_walk_and_a_new_state_checks_the_lists():
    # a force call marks the lists current; a cell walk re-sorts the atoms and a new
    # state replaces the positions: the next step must rebuild, as a fresh context does
    s = synth.electrolyte(2500, seed=68, charges="2:1", n_types=2)
    a, _ = make_ctx(s, rb.FP32, seed=6, thermostat=1)
    a.forces(1)
    a.rbl_lists(1)
    a.set_state_u(s.u, vel=s.v, step=0)
    a.step(3)
    b, _ = make_ctx(s, rb.FP32, seed=6, thermostat=1)
    b.set_state_u(s.u, vel=s.v, step=0)
    b.step(3)
    ua, va, _ = a.get_state_u()
    ub, vb, _ = b.get_state_u()
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    a.close()
    b.close()
