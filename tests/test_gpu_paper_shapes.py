"""GPU parity in the regimes of the paper's efficiency runs (Sec. 4.2), at
density 0.01 sigma^-3 and batch size p = 30:

  * the primitive 1:1 electrolyte: r_core = 6, r_cut = 12, alpha = 0.362,
    Bjerrum length 3.5 (coulomb_k), P = 100;
  * the uncharged LJ fluid, RBL only: r_core = 2.5, r_cut = 5.

Lists (|C|, N_s) and batches bit-exact against the oracle, forces within the
precision's tolerance; at the electrolyte benchmark's size (100,000 atoms) on a
sample of atoms.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

EL = dict(alpha=0.362, r_core=6.0, r_cut=12.0, rbl_p=30, rbe_P=100, coulomb_k=3.5)
LJ = dict(alpha=0.62, r_core=2.5, r_cut=5.0, rbl_p=30, rbe_P=10, coulomb_k=1.0, flags=rb.NO_RBE)


def _lj_fluid(n, seed):
    s = synth.electrolyte(n, seed=seed, charges="1:1", n_types=1, density=0.01)
    s.q = s.q * 0.0
    return s


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_primitive_electrolyte_density_001(prec):
    s = synth.electrolyte(2000, seed=91, charges="1:1", n_types=1, density=0.01)
    ctx, _ = make_ctx(s, prec, seed=8, **EL)
    for step in (0, 3):
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, EL["alpha"], EL["coulomb_k"],
                       EL["r_core"], EL["r_cut"], EL["rbl_p"], 8, step)
        assert np.array_equal(nc, o["n_core"]) and np.array_equal(ns, o["n_shell"])
        assert np.array_equal(b, o["batch"])
        assert ns.mean() > 30  # the shell is larger than the batch: p of N_s are drawn
        F = to_np(ctx.forces(step))
        Fo, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, EL["alpha"], EL["coulomb_k"],
                              EL["r_core"], EL["r_cut"], EL["rbl_p"], EL["rbe_P"], 8, step)
        assert rel_err(F, Fo) < TOL[prec], (step, rel_err(F, Fo))
    ctx.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_lj_fluid_density_001_rbl_only(prec):
    s = _lj_fluid(2000, 92)
    ctx, _ = make_ctx(s, prec, seed=9, **LJ)
    for step in (0, 5):
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, LJ["alpha"], 1.0, LJ["r_core"],
                       LJ["r_cut"], LJ["rbl_p"], 9, step)
        assert np.array_equal(nc, o["n_core"]) and np.array_equal(ns, o["n_shell"])
        assert np.array_equal(b, o["batch"])
        F = to_np(ctx.rbl_forces(step))
        Fo = o["F"] - o["Fsum"] / s.n
        assert rel_err(F, Fo) < TOL[prec], (step, rel_err(F, Fo))
        E = ctx.energy(step)
        assert abs(E["e_lj"] - o["E_lj"]) <= (1e-10 if prec == rb.FP64 else 1e-5) * abs(o["E_lj"])
        assert E["e_rbe"] == 0.0 and E["e_coul_real"] == 0.0
    ctx.close()


def test_primitive_electrolyte_benchmark_size_sample():
    import torch

    import bench

    saved = dict(bench.PARAMS)
    bench.PARAMS.update(bench.WORKLOADS["el001"]["params"])
    try:
        system = bench.make_system(100_000, 2, "el001")
        ctx = bench.make_ctx(system, rb.FP32, torch.device("cuda:0"))
        s = system.systems[0]
        sample = np.sort(np.random.default_rng(9).choice(s.n, 300, replace=False))
        step = 1
        nc, ns, b = (to_np(t).astype(np.int64) for t in ctx.rbl_lists(step))
        o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, EL["alpha"], EL["coulomb_k"],
                       EL["r_core"], EL["r_cut"], EL["rbl_p"], 2, step, sel=sample)
        assert np.array_equal(nc[sample], o["n_core"])
        assert np.array_equal(ns[sample], o["n_shell"])
        assert np.array_equal(b[sample], o["batch"])
        F = to_np(ctx.forces(step))[sample]
        Fr, _, _, _ = oracle.rbe_forces(s.u, s.q, s.L, EL["alpha"], EL["coulomb_k"], EL["rbe_P"], 2,
                                        step, sel=sample)
        Fo = Fr + o["F"] - o["Fsum"] / s.n
        assert rel_err(F, Fo) < TOL[rb.FP32], rel_err(F, Fo)
        ctx.close()
    finally:
        bench.PARAMS.clear()
        bench.PARAMS.update(saved)
