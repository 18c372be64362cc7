"""Tile shapes and the autotuner.

Every tile shape computes the same method: the modes, list counts and batches
stay bit-exact (they are integer work) and the forces stay within the
precision's tolerance of the FP64 oracle; only the rounding order of the
structure-factor sums and of the pair sums changes.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(1, 512, 64), (2, 2048, 128), (1, 1024, 256), (2, 512, 256)]


@pytest.fixture(scope="module")
def sys3k():
    return synth.electrolyte(3001, seed=21, charges="2:1", n_types=3)


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_every_tile_shape_matches_oracle(sys3k, prec):
    s = sys3k
    ctx, _ = make_ctx(s, prec, rbe_P=300, seed=5)
    Fo, Eo = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 300, 5, 1)
    nc0, ns0, b0 = (to_np(t) for t in ctx.rbl_lists(1))
    m0, _ = ctx.rbe_modes(1)
    for shape in SHAPES:
        ctx.set_tiles(*shape)
        assert ctx.tiles()[:3] == shape
        F = to_np(ctx.forces(1))
        assert rel_err(F, Fo) < TOL[prec], shape
        nc, ns, b = (to_np(t) for t in ctx.rbl_lists(1))
        assert np.array_equal(nc, nc0) and np.array_equal(ns, ns0) and np.array_equal(b, b0)
        m, _ = ctx.rbe_modes(1)
        assert np.array_equal(m, m0)
        E = ctx.energy(1)
        for k, ref in zip(("e_coul_real", "e_lj", "e_rbe"), Eo):
            assert abs(E[k] - ref) <= TOL[prec] * abs(ref) + 1e-12, (shape, k)
    ctx.close()


def test_set_tiles_rejects_other_values(sys3k):
    ctx, _ = make_ctx(sys3k, rb.FP32)
    for bad in [(0, 1024, 256), (3, 1024, 256), (2, 1000, 256), (2, 1024, 100)]:
        with pytest.raises(rb.RBMDError):
            ctx.set_tiles(*bad)
    assert ctx.tiles() == (2, 1024, 256, 0)
    ctx.close()


def test_autotune_keeps_a_valid_shape_and_the_dynamics(sys3k):
    import torch

    s = sys3k
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=100, seed=3, thermostat=1)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    ctx.step(2)  # captures the step graph with the default shape
    u0, v0, st0 = ctx.get_state_u()
    chosen = ctx.autotune(step=2)
    assert chosen == ctx.tiles()
    assert chosen[0] in (1, 2) and chosen[1] in (512, 1024, 2048) and chosen[2] in (64, 128, 256)
    assert chosen[3] in (0, 1)
    u1, v1, st1 = ctx.get_state_u()  # the state is untouched
    assert st1 == st0 and torch.equal(u0, u1) and torch.equal(v0, v1)
    ctx.step(2)  # re-captured with the chosen shape
    F = to_np(ctx.forces(9))
    u, _, _ = ctx.get_state_u()
    uu = (to_np(u).astype(np.int64) % 2 ** 32).astype(np.uint32)
    Fo, _ = oracle.forces(uu, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 100, 3, 9)
    assert rel_err(F, Fo) < TOL[rb.FP32]
    ctx.close()


def test_batch_with_tiles_equals_standalone():
    import torch

    systems = synth.replicas([1200, 2500], seed=6, charges="1:1")
    cat = synth.concat(systems)
    dev = torch.device("cuda:0")
    b = rb.RBMD(torch.from_numpy(cat["x"]).to(dev), torch.from_numpy(cat["q"]).to(dev),
                cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"], seed=[1, 2],
                replica=[0, 1], rbe_P=90)
    b.set_state_u(cat["u"], step=0)
    b.set_tiles(1, 512, 64)
    F = b.forces(4)
    off = 0
    for r, s in enumerate(systems):
        c, _ = make_ctx(s, rb.FP32, rbe_P=90, seed=r + 1, replica=r)
        c.set_tiles(1, 512, 64)
        assert torch.equal(F[off:off + s.n], c.forces(4))
        off += s.n
        c.close()
    b.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_pair_table_matches_oracle(sys3k, prec):
    """The look-up table replaces erfc/exp in the pair kernels: forces and energies
    stay within the precision's tolerance of the exact oracle; lists unchanged."""
    s = sys3k
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=8, flags=rb.PAIR_TABLE)
    assert ctx.tiles()[3] == 1
    Fo, Eo = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 100, 8, 3)
    F = to_np(ctx.forces(3))
    assert rel_err(F, Fo) < TOL[prec]
    E = ctx.energy(3)
    for k, ref in zip(("e_coul_real", "e_lj", "e_rbe"), Eo):
        assert abs(E[k] - ref) <= TOL[prec] * abs(ref) + 1e-12, k
    Fr = to_np(ctx.rbl_forces(3))
    ctx.set_pair_table(False)
    Fx = to_np(ctx.rbl_forces(3))
    # the two evaluations of the same short-range force agree to the table's accuracy
    assert rel_err(Fr, Fx) < (3e-6 if prec == rb.FP32 else 1e-11)
    ctx.close()


def test_pair_table_exact_lists_and_fallback(sys3k, monkeypatch):
    # the exact-list mode and the overflow fallback read the same table
    s = sys3k
    monkeypatch.setenv("RBMD_LIST_CAPS", "2,3")
    ctx, _ = make_ctx(s, rb.FP64, rbe_P=50, seed=9, flags=rb.PAIR_TABLE)
    F = to_np(ctx.rbl_forces(1))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 9, 1)
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < 1e-10
    ctx.close()
