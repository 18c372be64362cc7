"""GPU parity of the virial tensor and pressure (rbmd_energy) against the FP64
oracle, through the C ABI.

The virial is W_ab = -dE/d strain_ab at fixed fractional coordinates: the pair
part over the RBL lists with their weights (Eqs. 2, 10, 15) and the RBE
estimate of the Fourier part (Eq. 8 with the sampled modes of Eq. 12).  Both
sides draw the same modes and batches; tensors must agree within the force
tolerance of the precision (relative to the tensor's largest entry): the list
path, the exact-list mode, the overflow fallback, the pair look-up table, the
full Ewald mode list and a batch of replicas.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx

pytestmark = pytest.mark.gpu

PRECS = [rb.FP64, rb.FP32]


@pytest.fixture(scope="module")
def sys_2000():
    return synth.electrolyte(2011, seed=41, charges="2:1", n_types=3)


def _close(W, Wo, tol):
    scale = np.abs(Wo).max()
    return np.abs(np.asarray(W) - Wo).max() <= tol * scale


def _check(ctx, s, step, prec, seed, p=10, P=100, exact=False):
    E = ctx.energy(step)
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, p, seed, step,
                   exact=exact)
    Wk = oracle.rbe_virial(s.u, s.q, s.L, 0.62, 1.0, P, seed, step)
    tol = TOL[prec]
    assert abs(E["virial_coul_real"] - np.trace(o["W_coul"])) <= tol * abs(np.trace(o["W_coul"]))
    assert abs(E["virial_lj"] - np.trace(o["W_lj"])) <= tol * abs(np.trace(o["W_lj"]))
    assert abs(E["virial_rbe"] - np.trace(Wk)) <= tol * np.abs(Wk).max() * 3
    Wo = o["W_coul"] + o["W_lj"] + Wk
    assert _close(E["virial"], Wo, tol), (E["virial"], Wo)
    V = s.L ** 3
    p_ref = (2 * E["e_kinetic"] + np.trace(Wo)) / (3 * V)
    assert abs(E["pressure"] - p_ref) <= tol * (abs(p_ref) + 2 * E["e_kinetic"] / (3 * V))
    return E


@pytest.mark.parametrize("prec", PRECS)
def test_virial_matches_oracle(sys_2000, prec):
    s = sys_2000
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=6)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    for step in (0, 4):
        _check(ctx, s, step, prec, 6)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_virial_exact_lists(sys_2000, prec):
    s = sys_2000
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=6, flags=rb.RBL_EXACT)
    _check(ctx, s, 1, prec, 6, exact=True)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_virial_overflow_fallback(sys_2000, prec, monkeypatch):
    s = sys_2000
    monkeypatch.setenv("RBMD_LIST_CAPS", "3,7")
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=6)
    monkeypatch.delenv("RBMD_LIST_CAPS")
    _check(ctx, s, 2, prec, 6)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_virial_pair_table(sys_2000, prec):
    s = sys_2000
    ctx, _ = make_ctx(s, prec, rbe_P=100, seed=6, flags=rb.PAIR_TABLE)
    _check(ctx, s, 3, prec, 6)
    ctx.close()


@pytest.mark.parametrize("prec", PRECS)
def test_full_ewald_mode_virial(prec):
    s = synth.config1()
    ctx, _ = make_ctx(s, prec, flags=rb.FULL_EWALD_MODES | rb.RBL_EXACT)
    E = ctx.energy(0)
    M = oracle.sampler_M(s.L, 0.62)
    _, Wk = oracle.ewald_virial(s.u, s.q, s.L, 0.62, 1.0, 3.5, M)
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 0, 0, exact=True)
    Wo = Wk + o["W_coul"] + o["W_lj"]
    assert abs(E["virial_rbe"] - np.trace(Wk)) <= TOL[prec] * np.abs(Wk).max() * 3
    assert _close(E["virial"], Wo, TOL[prec])
    ctx.close()


def test_virial_of_batched_replicas():
    # replica r of a batch has the virial of a stand-alone context, bit for bit
    sizes = [700, 1500, 950]
    reps = [synth.electrolyte(n, seed=50 + r, charges="1:1", n_types=1) for r, n in enumerate(sizes)]
    import torch

    dev = torch.device("cuda:0")
    cat = lambda k: np.concatenate([getattr(x, k) for x in reps])
    pos = torch.from_numpy(np.concatenate([x.x for x in reps])).to(dev, torch.float32)
    q = torch.from_numpy(cat("q")).to(dev, torch.float32)
    vel = torch.from_numpy(cat("v")).to(dev, torch.float32)
    ctx = rb.RBMD(pos, q, reps[0].eps, reps[0].sig, box_length=[x.L for x in reps],
                  n_atoms=sizes, seed=[3, 4, 5], replica=[0, 1, 2], precision=rb.FP32,
                  rbe_P=60, vel=vel)
    ctx.set_state_u(cat("u"), step=0)
    Eb = ctx.energy_batch(1)
    for r, x in enumerate(reps):
        c, _ = make_ctx(x, rb.FP32, rbe_P=60, seed=3 + r, replica=r)
        E = c.energy(1)
        assert np.array_equal(E["virial"], Eb[r]["virial"])
        assert E["pressure"] == Eb[r]["pressure"]
        c.close()
    ctx.close()
