"""GPU adjoint (rbmd_energy_backward) against the oracle's gradients, finite
differences and the forces.

Gradients of E = E_coul_real + E_lj + E_rbe + E_self with the draws of the step
held fixed: positions, charges and per-type LJ epsilon and sigma.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

KW = dict(rbe_P=60, rbl_p=10, seed=8, coulomb_k=1.0)


@pytest.fixture(scope="module")
def sys_g():
    return synth.electrolyte(1537, seed=23, charges="2:1", n_types=3)


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_gradients_match_oracle(sys_g, prec):
    s = sys_g
    ctx, _ = make_ctx(s, prec, **KW)
    step = 3
    dpos, dq, de, ds = ctx.energy_backward(step, 1.0)
    E, dr_o, dq_o, de_o, ds_o = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0,
                                                   2.0, 3.5, 10, 60, 8, step)
    tol = TOL[prec]
    assert rel_err(to_np(dpos), dr_o) < tol
    assert rel_err(to_np(dq), dq_o) < tol
    assert rel_err(de, de_o) < 10 * tol
    assert rel_err(ds, ds_o) < 10 * tol
    En = ctx.energy(step)
    assert abs(En["e_potential"] - E.sum()) < (1e-10 if prec == rb.FP64 else 1e-5) * abs(E.sum())
    # grad_out scales every output
    dpos2, dq2, de2, ds2 = ctx.energy_backward(step, -2.5)
    assert rel_err(to_np(dpos2), -2.5 * to_np(dpos)) < 1e-6
    assert rel_err(de2, -2.5 * np.asarray(de)) < 1e-6
    ctx.close()


def test_exact_lists_gradient_is_minus_force(sys_g):
    s = sys_g
    ctx, _ = make_ctx(s, rb.FP64, flags=rb.RBL_EXACT, **KW)
    dpos, *_ = ctx.energy_backward(1, 1.0)
    F_rbl = to_np(ctx.rbl_forces(1))
    E = ctx.energy(1)
    fcorr = -np.asarray(E["fsum_short"]) / s.n
    F = F_rbl - fcorr + to_np(ctx.rbe_forces(1))
    assert rel_err(-to_np(dpos), F) < 1e-10
    ctx.close()


def test_fp64_gradients_pass_finite_differences(sys_g):
    import torch

    s = sys_g
    ctx, _ = make_ctx(s, rb.FP64, **KW)
    step = 5
    dpos, dq, de, ds = ctx.energy_backward(step, 1.0)
    dpos, dq = to_np(dpos), to_np(dq)
    base_lists = [to_np(t) for t in ctx.rbl_lists(step)]
    rng = np.random.default_rng(0)
    u0 = s.u.astype(np.int64)
    done = 0
    for trial in range(8):
        # exact integer displacement of every coordinate, about 1e-5 sigma
        du = np.rint(rng.normal(size=u0.shape) * 1e-5 * 2.0 ** 32 / s.L).astype(np.int64)
        dx = du * (s.L / 2.0 ** 32)
        es = []
        ok = True
        for sgn in (1, -1):
            ctx.set_state_u(((u0 + sgn * du) % 2 ** 32).astype(np.uint32), step=step)
            if any(not np.array_equal(a, to_np(b)) for a, b in zip(base_lists, ctx.rbl_lists(step))):
                ok = False
            es.append(ctx.energy(step)["e_potential"])
        if not ok:
            continue
        fd = (es[0] - es[1]) / 2.0
        an = float(np.sum(dpos * dx))
        assert abs(fd - an) <= 1e-4 * (abs(an) + 1e-6), (fd, an)
        done += 1
    assert done >= 3
    ctx.set_state_u(s.u, step=step)
    h = 1e-6
    # charges: neutral perturbation direction, lists unaffected
    w = rng.normal(size=s.n)
    w -= w.mean()
    w /= np.linalg.norm(w)
    es = []
    for sgn in (1, -1):
        ctx.set_charges(torch.from_numpy(s.q + sgn * h * w).cuda())
        es.append(ctx.energy(step)["e_potential"])
    ctx.set_charges(torch.from_numpy(s.q).cuda())
    fd = (es[0] - es[1]) / (2 * h)
    assert abs(fd - float(np.dot(dq, w))) <= 1e-4 * (abs(fd) + 1e-3)
    # per-type epsilon and sigma
    for t in range(len(s.eps)):
        for which, g in (("eps", de), ("sig", ds)):
            es = []
            for sgn in (1, -1):
                e2, s2 = s.eps.copy(), s.sig.copy()
                (e2 if which == "eps" else s2)[t] += sgn * h
                ctx.set_lj(e2, s2)
                es.append(ctx.energy(step)["e_potential"])
            fd = (es[0] - es[1]) / (2 * h)
            assert abs(fd - g[t]) <= 1e-4 * (abs(g[t]) + 1e-3), (which, t, fd, g[t])
    ctx.close()


def test_autograd_function():
    import torch
    from paper_2407_09315_b300.autograd import energy

    s = synth.electrolyte(900, seed=24, charges="1:1", n_types=2)
    ctx, _ = make_ctx(s, rb.FP64, **KW)
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(s.x).to(dev).requires_grad_(True)
    q = torch.from_numpy(s.q).to(dev).requires_grad_(True)
    eps = torch.tensor(s.eps, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(s.sig, dtype=torch.float64, requires_grad=True)
    E = energy(ctx, 2, pos, q, eps, sig)
    E.backward()
    ref = ctx.energy_backward(2, 1.0)
    assert rel_err(to_np(pos.grad), to_np(ref[0])) < 1e-12
    assert rel_err(to_np(q.grad), to_np(ref[1])) < 1e-12
    assert rel_err(eps.grad.numpy(), ref[2]) < 1e-12
    assert rel_err(sig.grad.numpy(), ref[3]) < 1e-12
    ctx.close()


def test_backward_grows_overflowing_lists(monkeypatch):
    s = synth.electrolyte(1200, seed=25, charges="2:1", n_types=2)
    monkeypatch.setenv("RBMD_LIST_CAPS", "2,5")
    ctx, _ = make_ctx(s, rb.FP64, **KW)
    monkeypatch.delenv("RBMD_LIST_CAPS")
    dpos, dq, de, ds = ctx.energy_backward(4, 1.0)
    E, dr_o, dq_o, de_o, ds_o = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0,
                                                   2.0, 3.5, 10, 60, 8, 4)
    assert rel_err(to_np(dpos), dr_o) < 1e-10
    assert rel_err(ds, ds_o) < 1e-9
    # the step graph still runs after the lists were reallocated
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(2)
    ctx.sync()
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_backward_after_energy_reuses_lists_and_modes(sys_g, prec):
    """rbmd_energy_backward right after rbmd_energy of the same state and step reuses
    the forward's lists, modes and structure factors; the gradients are the same bits
    as a backward that builds its own (another call in between clears the reuse), and
    two backward passes agree bit for bit (the reverse batches are summed in a fixed
    order)."""
    s = sys_g
    ctx, _ = make_ctx(s, prec, **KW)
    step = 4
    ctx.rbe_modes(step + 1)  # other modes in the arrays: nothing to reuse
    ctx.rbl_lists(step + 1)
    cold = [g if isinstance(g, np.ndarray) else to_np(g) for g in ctx.energy_backward(step, 1.0)]
    again = [g if isinstance(g, np.ndarray) else to_np(g) for g in ctx.energy_backward(step, 1.0)]
    ctx.energy(step)
    warm = [g if isinstance(g, np.ndarray) else to_np(g) for g in ctx.energy_backward(step, 1.0)]
    ctx.energy(step + 1)  # a forward of another step is not reused for this one
    other = [g if isinstance(g, np.ndarray) else to_np(g) for g in ctx.energy_backward(step, 1.0)]
    for a, b, c, d in zip(cold, again, warm, other):
        assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)
    ctx.close()
