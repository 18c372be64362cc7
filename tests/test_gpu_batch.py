"""Batched replicas: R independent systems stepped by one context.

The per-system arithmetic of a batch is the stand-alone arithmetic (same cells,
same 128/256-atom block partition, same tile partition of the structure factor,
same replica-local Philox counters), so every per-replica result must equal the
stand-alone context's bit for bit: modes, list counts, batches (ids shifted by
the replica's offset), forces, energies, gradients and trajectories.  One
replica is also checked against the FP64 oracle directly, and the batch draws
against the oracle's sampler.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import DEFAULTS, TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu

SIZES = [1000, 1537, 3001, 257]
SEEDS = [11, 12, 13, 14]
REPS = [0, 1, 2, 7]
T0S = [1.0, 1.5, 0.7, 1.2]


@pytest.fixture(scope="module")
def systems():
    return synth.replicas(SIZES, seed=4, charges="2:1", n_types=3, T0=T0S)


def make_batch(systems, precision, **kw):
    import torch

    dt = torch.float64 if precision == rb.FP64 else torch.float32
    cat = synth.concat(systems)
    prm = dict(DEFAULTS)
    prm.update(kw)
    dev = torch.device("cuda:0")
    ctx = rb.RBMD(torch.from_numpy(cat["x"]).to(dev, dt), torch.from_numpy(cat["q"]).to(dev, dt),
                  cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"],
                  precision=precision, vel=torch.from_numpy(cat["v"]).to(dev, dt),
                  types=torch.from_numpy(cat["types"]).to(dev), **prm)
    ctx.set_state_u(cat["u"], vel=cat["v"], step=0)
    return ctx


def solo(s, precision, r, **kw):
    kw = dict(kw)
    kw["seed"] = SEEDS[r]
    kw["replica"] = REPS[r]
    if "temperature" in kw:
        kw["temperature"] = T0S[r]
    ctx, _ = make_ctx(s, precision, **kw)
    ctx.set_state_u(s.u, vel=s.v, step=0)
    return ctx


def slices(n):
    off = np.concatenate([[0], np.cumsum(n)])
    return [slice(int(off[r]), int(off[r + 1])) for r in range(len(n))]


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_batch_forces_equal_standalone(systems, prec):
    import torch

    b = make_batch(systems, prec, seed=SEEDS, replica=REPS, rbe_P=120)
    for step in (0, 5):
        Fb = {k: getattr(b, k)(step).clone() for k in ("rbe_forces", "rbl_forces", "forces")}
        torch.cuda.synchronize()
        for r, (s, sl) in enumerate(zip(systems, slices(SIZES))):
            c = solo(s, prec, r, rbe_P=120)
            for k, F in Fb.items():
                Fs = getattr(c, k)(step)
                assert torch.equal(F[sl], Fs), (k, r, step)
            c.close()
    b.close()


def test_batch_draws_and_lists(systems):
    b = make_batch(systems, rb.FP32, seed=SEEDS, replica=REPS, rbe_P=64)
    assert b.R == len(SIZES) and rb.lib().rbmd_replica_count(b._h) == len(SIZES)
    step = 3
    m, rho = b.rbe_modes(step)
    nc, ns, bt = (to_np(t).astype(np.int64) for t in b.rbl_lists(step))
    for r, (s, sl) in enumerate(zip(systems, slices(SIZES))):
        mo = oracle.rbe_sample(SEEDS[r], step, 64, s.L, 0.62, replica=REPS[r])
        assert np.array_equal(m[64 * r:64 * (r + 1)], mo), r
        c = solo(s, rb.FP32, r, rbe_P=64)
        nc1, ns1, b1 = (to_np(t).astype(np.int64) for t in c.rbl_lists(step))
        assert np.array_equal(nc[sl], nc1) and np.array_equal(ns[sl], ns1), r
        shifted = np.where(bt[sl] >= 0, bt[sl] - sl.start, -1)
        assert np.array_equal(shifted, b1), r
        # ids of a replica's batch never leave the replica
        assert np.all((bt[sl] == -1) | ((bt[sl] >= sl.start) & (bt[sl] < sl.stop)))
        c.close()
    b.close()


def test_batch_replica_matches_oracle(systems):
    b = make_batch(systems, rb.FP64, seed=SEEDS, replica=REPS, rbe_P=100)
    F = to_np(b.forces(2))
    for r in (1, 3):
        s = systems[r]
        sl = slices(SIZES)[r]
        Fo, Eo = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 100,
                               SEEDS[r], 2, replica=REPS[r])
        assert rel_err(F[sl], Fo) < TOL[rb.FP64], r
        E = b.energy_batch(2)[r]
        for k, ref in zip(("e_coul_real", "e_lj", "e_rbe", "e_self"), Eo):
            assert abs(E[k] - ref) <= 1e-10 * abs(ref) + 1e-12, (r, k, E[k], ref)
    b.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_batch_energies_equal_standalone(systems, prec):
    b = make_batch(systems, prec, seed=SEEDS, replica=REPS, rbe_P=80)
    with pytest.raises(rb.RBMDError):
        b.energy(1)  # one set of terms is ambiguous for a batch
    Eb = b.energy_batch(1)
    for r, s in enumerate(systems):
        c = solo(s, prec, r, rbe_P=80)
        E = c.energy(1)
        for k in ("e_coul_real", "e_lj", "e_rbe", "e_self", "e_potential", "e_kinetic",
                  "temperature", "S", "fsum_short"):
            assert Eb[r][k] == E[k], (r, k, Eb[r][k], E[k])
        c.close()
    b.close()


@pytest.mark.parametrize("thermostat", [0, 1, 2, 3, 4])
def test_batch_trajectory_equals_standalone(systems, thermostat):
    import torch

    kw = dict(rbe_P=50, dt=0.002, thermostat=thermostat, temperature=1.0, tau_T=0.05)
    b = make_batch(systems, rb.FP32, seed=SEEDS, replica=REPS,
                   **{**kw, "temperature": T0S})
    b.step(2)
    b.step(3)  # the second call replays the captured step graph
    ub, vb, st = b.get_state_u()
    assert st == 5
    for r, (s, sl) in enumerate(zip(systems, slices(SIZES))):
        c = solo(s, rb.FP32, r, **kw)
        c.step(5)
        u1, v1, _ = c.get_state_u()
        assert torch.equal(ub[sl], u1) and torch.equal(vb[sl], v1), r
        c.close()
    b.close()


def test_batch_backward_equals_standalone(systems):
    import torch

    b = make_batch(systems, rb.FP64, seed=SEEDS, replica=REPS, rbe_P=60)
    dpos, dq, de, ds = b.energy_backward(4)
    de_sum = np.zeros_like(de)
    ds_sum = np.zeros_like(ds)
    for r, (s, sl) in enumerate(zip(systems, slices(SIZES))):
        c = solo(s, rb.FP64, r, rbe_P=60)
        p1, q1, e1, s1 = c.energy_backward(4)
        assert torch.equal(dpos[sl], p1) and torch.equal(dq[sl], q1), r
        de_sum += e1
        ds_sum += s1
        c.close()
    assert np.allclose(de, de_sum, rtol=1e-12, atol=1e-12)
    assert np.allclose(ds, ds_sum, rtol=1e-12, atol=1e-12)
    b.close()


def test_batch_each_replica_must_be_neutral(systems):
    import torch

    a = synth.electrolyte(100, seed=1, charges="1:1", lj=(systems[0].eps, systems[0].sig))
    c = synth.electrolyte(120, seed=2, charges="1:1", lj=(systems[0].eps, systems[0].sig))
    a.q[0] += 1.0
    c.q[0] -= 1.0  # the batch as a whole stays neutral
    cat = synth.concat([a, c])
    dev = torch.device("cuda:0")
    with pytest.raises(rb.RBMDError) as e:
        rb.RBMD(torch.from_numpy(cat["x"]).to(dev), torch.from_numpy(cat["q"]).to(dev),
                cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"])
    assert e.value.code == 2  # RBMD_ERR_NOT_NEUTRAL
