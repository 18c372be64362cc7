"""Parity at the benchmark's full size (the 1M-atom 2:1 electrolyte, P = 200, p = 10)
in the launch configuration bench.py times (its context, autotuned tiles, the
integrator's step graph): modes and lists bit-exact, and forces and energies of a
seeded sample of atoms against the oracle, which computes them one by one (the
momentum correction and the energies over all atoms).  Both the FP32 path and the
plain FP64 path its speed-up is quoted against (with the FP64 leg's own autotuned
shape, which picks the pair look-up table) are checked."""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb

from gpu_util import TOL, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch

    import bench

    system = bench.make_system(1_000_000, 2, "c3")
    ctx = bench.make_ctx(system, rb.FP32, torch.device("cuda:0"))
    ctx.autotune(step=0)
    yield bench.PARAMS, system.systems[0], ctx
    ctx.close()


@pytest.fixture(scope="module")
def setup64():
    import torch

    import bench

    system = bench.make_system(1_000_000, 2, "c3")
    ctx = bench.make_ctx(system, rb.FP64, torch.device("cuda:0"))
    ctx.autotune(step=0)
    yield bench.PARAMS, system.systems[0], ctx
    ctx.close()


def _check_state(prm, s, u, ctx, step, sample, prec=rb.FP32):
    # modes of the step, bit for bit
    m, _ = ctx.rbe_modes(step)
    mo = oracle.rbe_sample(2, step, prm["rbe_P"], s.L, prm["alpha"])
    assert np.array_equal(m, mo)
    # lists and batch of the sample, bit for bit
    nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
    o = oracle.rbl(u, s.q, s.types, s.eps, s.sig, s.L, prm["alpha"], prm["coulomb_k"],
                   prm["r_core"], prm["r_cut"], prm["rbl_p"], 2, step, sel=sample)
    assert np.array_equal(nc[sample], o["n_core"])
    assert np.array_equal(ns[sample], o["n_shell"])
    assert np.array_equal(b[sample], o["batch"])
    # total force of the sample: RBE + RBL + the correction over all atoms
    F = to_np(ctx.forces(step))[sample]
    Fr, Er, _, _ = oracle.rbe_forces(u, s.q, s.L, prm["alpha"], prm["coulomb_k"], prm["rbe_P"], 2,
                                     step, sel=sample)
    Fo = Fr + o["F"] - o["Fsum"] / s.n
    assert rel_err(F, Fo) < TOL[prec], rel_err(F, Fo)
    E = ctx.energy(step)
    for k, ref in (("e_coul_real", o["E_coul"]), ("e_lj", o["E_lj"]), ("e_rbe", Er)):
        assert abs(E[k] - ref) <= TOL[prec] * abs(ref), (k, E[k], ref)


def test_full_size_initial_state(setup):
    prm, s, ctx = setup
    sample = np.sort(np.random.default_rng(5).choice(s.n, 400, replace=False))
    _check_state(prm, s, s.u, ctx, 0, sample)


def test_full_size_after_steps(setup):
    prm, s, ctx = setup
    ctx.step(3)  # the step graph bench.py times
    u, _, st = ctx.get_state_u()
    assert st == 3
    u = (to_np(u).astype(np.int64) % 2 ** 32).astype(np.uint32)
    # every atom moved, none by more than a small fraction of the box
    d = (u.astype(np.int64) - s.u.astype(np.int64) + 2 ** 31) % 2 ** 32 - 2 ** 31
    assert np.abs(d).max() < 2 ** 32 // 1000
    sample = np.sort(np.random.default_rng(6).choice(s.n, 400, replace=False))
    _check_state(prm, s, u, ctx, 3, sample)


def test_full_size_fp64_path(setup64):
    prm, s, ctx = setup64
    assert ctx.tiles()[3] in (0, 1)
    sample = np.sort(np.random.default_rng(7).choice(s.n, 200, replace=False))
    _check_state(prm, s, s.u, ctx, 0, sample, rb.FP64)
    ctx.step(2)
    u, _, st = ctx.get_state_u()
    assert st == 2
    u = (to_np(u).astype(np.int64) % 2 ** 32).astype(np.uint32)
    _check_state(prm, s, u, ctx, 2, sample, rb.FP64)
