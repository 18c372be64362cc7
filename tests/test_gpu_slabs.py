"""Spatial decomposition on the GPU (slab contexts, rbmd_init_slab): the ranks of a
decomposition emulated as contexts in one process on one device (they never
wait on one another, so no collective is needed here; the exchanges are the
host-side sums of paper_2407_09315_b300.slabs).

  * the slab contexts' exact partial structure factors add up, bit for bit, to
    those of one context holding every atom when the atom tiles hold the same
    atoms (slab 0 owning a whole number of 1024-atom tiles, atoms ordered by
    slab), and their RBE forces are then bit-identical;
  * the lists (|C|, N_s) and batches of every owned atom equal the one-context
    lists and the oracle's (the draws are keyed by global ids);
  * the distributed total force (RBE + RBL + the correction summed over ranks)
    matches the one-context force and the oracle within the precision's
    tolerance, for two tile-aligned slabs and for three equal slabs.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import slabs, synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

PRM = dict(alpha=0.62, r_core=2.0, r_cut=3.5, rbl_p=10, rbe_P=120, coulomb_k=1.0, seed=11)


def _system_by_slab(n, seed, n0):
    """A system whose atoms are ordered by slab, slab 0 holding the n0 atoms of
    smallest x; returns (system, bounds)."""
    s = synth.electrolyte(n, seed=seed, charges="1:1", n_types=2)
    order = np.argsort(s.u[:, 0], kind="stable")
    s = synth.System(L=s.L, u=np.ascontiguousarray(s.u[order]), q=s.q[order],
                     types=s.types[order], eps=s.eps, sig=s.sig, v=s.v[order])
    b = int(s.u[n0, 0])
    assert int(s.u[n0 - 1, 0]) < b
    return s, [0, b, 1 << 32]


def _ranks(s, prec, bounds, n_ranks):
    import torch

    owned, halo = slabs.slab_partition(s.u, s.L, n_ranks, PRM["r_cut"], bounds=bounds)
    kw = {k: v for k, v in PRM.items()}
    return [slabs.SlabRank(s.u, s.q, s.types, s.eps, s.sig, s.L, owned[r], halo[r],
                           precision=prec, device=torch.device("cuda:0"), **kw)
            for r in range(n_ranks)]


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_two_slabs_bit_exact_structure_factors(prec):
    s, bounds = _system_by_slab(8192, 111, 4096)
    ranks = _ranks(s, prec, bounds, 2)
    assert [r.n_owned for r in ranks] == [4096, 4096]
    one, _ = make_ctx(s, prec, **PRM)
    for step in (0, 3):
        acc1 = one.rho_partial(step)
        parts = [r.ctx.rho_partial(step) for r in ranks]
        tot = np.zeros_like(acc1)
        for a in parts:
            rb.rho_acc_add(tot, a)
        assert np.array_equal(tot, acc1), step
        # same sums -> the same RBE forces, bit for bit
        F1 = to_np(one.rbe_forces(step))
        for r in ranks:
            Fr = to_np(r.ctx.forces_rho(step, tot))[: r.n_owned]
            assert np.array_equal(Fr, F1[r.owned]), step
    one.close()
    for r in ranks:
        r.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
@pytest.mark.parametrize("n_ranks", [2, 3])
def test_distributed_forces_match_one_context_and_oracle(prec, n_ranks):
    if n_ranks == 2:
        s, bounds = _system_by_slab(8192, 112, 4096)
    else:
        s = synth.electrolyte(6001, seed=113, charges="2:1", n_types=2)
        bounds = None
    ranks = _ranks(s, prec, bounds, n_ranks)
    one, _ = make_ctx(s, prec, **PRM)
    step = 2
    F, _ = slabs.slab_forces_local(ranks, step)
    F1 = to_np(one.forces(step))
    assert rel_err(F, F1) < TOL[prec], rel_err(F, F1)
    Fo, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, PRM["alpha"], PRM["coulomb_k"],
                          PRM["r_core"], PRM["r_cut"], PRM["rbl_p"], PRM["rbe_P"], PRM["seed"], step)
    assert rel_err(F, Fo) < TOL[prec], rel_err(F, Fo)
    # lists and batches of the owned atoms: the one-context lists, in global ids
    nc1, ns1, b1 = (to_np(t).astype(np.int64) for t in one.rbl_lists(step))
    for r in ranks:
        nc, ns, b = (to_np(t).astype(np.int64) for t in r.ctx.rbl_lists(step))
        o = r.n_owned
        assert np.array_equal(nc[:o], nc1[r.owned]) and np.array_equal(ns[:o], ns1[r.owned])
        bg = np.where(b[:o] >= 0, r.rows[np.maximum(b[:o], 0)], -1)
        bg = np.sort(np.where(bg < 0, np.iinfo(np.int64).max, bg), axis=1)
        bg = np.where(bg == np.iinfo(np.int64).max, -1, bg)
        assert np.array_equal(bg, b1[r.owned])
    one.close()
    for r in ranks:
        r.close()


def test_slab_context_rejects_unsupported_calls():
    s, bounds = _system_by_slab(4096, 114, 2048)
    ranks = _ranks(s, rb.FP32, bounds, 2)
    with pytest.raises(rb.RBMDError):
        ranks[0].ctx.step(1)
    with pytest.raises(rb.RBMDError):
        ranks[0].ctx.energy(0)
    for r in ranks:
        r.close()
