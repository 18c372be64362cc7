"""Batch sizes above 32 (the paper's p = 100, Sec. 4.1): the warp-sorted selection
gives the same lists and batches as the oracle, bit for bit, and the same forces
within tolerance; atoms with N_s <= p and N_s > p are both covered."""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

# the paper's LJ/electrolyte accuracy box: r_c = 2.5, r_s = 5, Bjerrum length 3.5,
# alpha = 0.362, p = 100, at about unit density (N = 1000, L = 10.2 > 2 r_s)
KW = dict(alpha=0.362, r_core=2.5, r_cut=5.0, coulomb_k=3.5, rbe_P=100)


@pytest.fixture(scope="module")
def dense():
    return synth.electrolyte(1000, L=10.2, seed=31, charges="1:1", n_types=1, dmin_factor=0.7)


@pytest.fixture(scope="module")
def mixed():
    # shell counts around 46: some atoms keep their whole shell, some select
    return synth.electrolyte(3000, density=0.1, seed=32, charges="1:1", n_types=2,
                             dmin_factor=0.7)


@pytest.mark.parametrize("which,p", [("dense", 100), ("mixed", 46), ("mixed", 33)])
def test_lists_bit_exact(which, p, request):
    s = request.getfixturevalue(which)
    ctx, _ = make_ctx(s, rb.FP32, rbl_p=p, seed=7, **KW)
    for step in (0, 5):
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.362, 3.5, 2.5, 5.0, p, 7, step)
        assert np.array_equal(nc, o["n_core"]) and np.array_equal(ns, o["n_shell"])
        assert np.array_equal(b, o["batch"]), step
        if which == "mixed":
            assert (ns > p).any() and (ns <= p).any()
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_forces_match_oracle(dense, prec):
    s = dense
    ctx, _ = make_ctx(s, prec, rbl_p=100, seed=7, **KW)
    F = to_np(ctx.rbl_forces(2))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.362, 3.5, 2.5, 5.0, 100, 7, 2)
    assert rel_err(F, o["F"] - o["Fsum"] / s.n) < TOL[prec]
    ctx.close()


def test_gradients_with_large_batch(mixed):
    s = mixed
    ctx, _ = make_ctx(s, rb.FP64, rbl_p=40, seed=9, **KW)
    dpos, dq, de, ds = ctx.energy_backward(1)
    E, dr_o, dq_o, de_o, ds_o = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.362,
                                                   3.5, 2.5, 5.0, 40, 100, 9, 1)
    assert rel_err(to_np(dpos), dr_o) < 1e-10
    assert rel_err(to_np(dq), dq_o) < 1e-10
    assert rel_err(de, de_o) < 1e-9
    ctx.close()


def test_batch_size_limits():
    s = synth.electrolyte(500, seed=33, charges="1:1")
    with pytest.raises(rb.RBMDError):
        make_ctx(s, rb.FP32, rbl_p=1025)
    ctx, _ = make_ctx(s, rb.FP32, rbl_p=1024)  # larger than every shell: whole shells
    nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(0))
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 1024, 0, 0)
    assert np.array_equal(b, o["batch"])
    ctx.close()
