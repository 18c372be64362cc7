"""Degenerate and edge cases of the GPU path against the oracle: a box too small for
the 5x5x5 stencil (every cell of an axis, once), two atoms, a single neutral atom,
an uncharged LJ fluid (RBE force zero), the exact-list mode at p = 1."""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cell_div", [1, 2])
def test_small_box_uses_every_cell_once(cell_div):
    s = synth.electrolyte(100, seed=41, charges="1:1", n_types=2)  # L = 7.94: < 5 cells
    assert s.L < 2 * 5 * 3.5 / 2
    ctx, _ = make_ctx(s, rb.FP64, seed=3, cell_div=cell_div, rbe_P=30)
    nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(1))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 3, 1)
    assert np.array_equal(nc, o["n_core"]) and np.array_equal(ns, o["n_shell"])
    assert np.array_equal(b, o["batch"])
    F = to_np(ctx.forces(1))
    Fo, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 30, 3, 1)
    assert rel_err(F, Fo) < TOL[rb.FP64]
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_two_atoms(prec):
    import torch

    L = 8.0
    x = np.array([[1.0, 1.0, 1.0], [2.2, 1.3, 0.9]])
    q = np.array([1.0, -1.0])
    dev = torch.device("cuda:0")
    dt = torch.float64 if prec == rb.FP64 else torch.float32
    ctx = rb.RBMD(torch.from_numpy(x).to(dev, dt), torch.from_numpy(q).to(dev, dt), [1.0], [1.0],
                  box_length=L, precision=prec, rbe_P=20, seed=1)
    u, _, _ = ctx.get_state_u()
    u = (to_np(u).astype(np.int64) % 2 ** 32).astype(np.uint32)
    F = to_np(ctx.forces(0))
    Fo, _ = oracle.forces(u, q, np.zeros(2, np.int32), [1.0], [1.0], L, 0.62, 1.0, 2.0, 3.5, 10,
                          20, 1, 0)
    assert rel_err(F, Fo) < TOL[prec]
    assert np.allclose(F[0], -F[1], rtol=1e-6, atol=1e-9)  # Newton's third law for one pair
    ctx.close()


def test_single_neutral_atom_steps():
    import torch

    dev = torch.device("cuda:0")
    x = torch.tensor([[1.0, 2.0, 3.0]], device=dev)
    v = torch.tensor([[0.5, -0.25, 1.0]], device=dev)
    ctx = rb.RBMD(x, torch.zeros(1, device=dev), [1.0], [1.0], box_length=8.0, vel=v,
                  thermostat=1, rbe_P=10)
    F = to_np(ctx.forces(0))
    assert np.all(F == 0)
    ctx.step(5)
    _, v1, st = ctx.get_state()
    assert st == 5 and torch.allclose(v1, v)  # free flight, no thermostat for one atom
    ctx.close()


def test_uncharged_fluid_has_no_rbe_force():
    s = synth.electrolyte(800, seed=42, charges="1:1", n_types=2)
    s.q[:] = 0.0
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=50, seed=4)
    assert np.all(to_np(ctx.rbe_forces(2)) == 0)
    F = to_np(ctx.forces(2))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 4, 2)
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[rb.FP32]
    E = ctx.energy(2)
    assert E["e_rbe"] == 0.0 and E["e_coul_real"] == 0.0 and E["e_self"] == 0.0
    ctx.close()


def test_batch_of_one():
    s = synth.electrolyte(1500, seed=43, charges="2:1", n_types=2)
    ctx, _ = make_ctx(s, rb.FP64, rbl_p=1, seed=5)
    nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(0))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 1, 5, 0)
    assert np.array_equal(b, o["batch"])
    F = to_np(ctx.rbl_forces(0))
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[rb.FP64]
    ctx.close()
