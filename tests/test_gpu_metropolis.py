"""Metropolis mode chains (RBMD_METROPOLIS_MODES, Algorithm 1 step 1) on the GPU
against the oracle's chains: modes bit-exact at every step (advancing, replaying
from step 0, inside the step graph, per replica of a batch), and the RBE force of
those modes within tolerance."""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s2k():
    return synth.electrolyte(2000, seed=51, charges="2:1", n_types=2)


def test_chains_bit_exact_forward_and_replay(s2k):
    s = s2k
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=150, seed=77, replica=2, flags=rb.METROPOLIS_MODES,
                      mh_moves=5)
    for step in (0, 1, 5, 3, 9, 9, 0):
        m, _ = ctx.rbe_modes(step)
        mo = oracle.rbe_metropolis(77, step, 150, s.L, 0.62, 5, replica=2)
        assert np.array_equal(m, mo), step
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_rbe_force_of_the_chains(s2k, prec):
    s = s2k
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=5, flags=rb.METROPOLIS_MODES)
    F = to_np(ctx.rbe_forces(4))
    m = oracle.rbe_metropolis(5, 4, 100, s.L, 0.62, 8)
    W = np.full(100, oracle.rbe_S(s.L, 0.62) / 100)
    Fo, Eo, _ = oracle.mode_forces(s.u, s.q, s.L, 1.0, m, W)
    assert rel_err(F, Fo) < TOL[prec]
    assert abs(ctx.energy(4)["e_rbe"] - Eo) <= TOL[prec] * abs(Eo)
    ctx.close()


def test_chains_in_the_step_graph_and_batches():
    systems = synth.replicas([1500, 2500], seed=8, charges="1:1")
    cat = synth.concat(systems)
    import torch

    dev = torch.device("cuda:0")
    b = rb.RBMD(torch.from_numpy(cat["x"]).to(dev), torch.from_numpy(cat["q"]).to(dev),
                cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"], seed=[3, 4],
                replica=[0, 1], rbe_P=64, flags=rb.METROPOLIS_MODES, mh_moves=3)
    b.set_state_u(cat["u"], step=0)
    b.step(2)
    b.step(3)  # graph replays advance the chains by one step each
    m, _ = b.rbe_modes(5)
    for r, s in enumerate(systems):
        mo = oracle.rbe_metropolis(3 + r, 5, 64, s.L, 0.62, 3, replica=r)
        assert np.array_equal(m[64 * r:64 * (r + 1)], mo), r
    b.close()


def test_metropolis_with_full_modes_is_invalid(s2k):
    with pytest.raises(rb.RBMDError):
        make_ctx(s2k, rb.FP32, flags=rb.METROPOLIS_MODES | rb.FULL_EWALD_MODES)
