"""The two-stream force evaluation.

A force evaluation runs the RBE sampling and structure factors (Algorithm 1
steps 1-2) on a second stream beside the cell sort and the RBL kernels
(Algorithm 2), and joins them before the RBE force pass; an energy evaluation
runs its RBE part (with the mode sums) there too.  The two parts share
no buffer, so the result must be the one-stream result bit for bit:
trajectories, forces and energies, for one system and for a batch.
RBMD_ONE_STREAM=1 at context creation selects the one-stream evaluation.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sys5k():
    return synth.electrolyte(5003, seed=31, charges="2:1", n_types=3)


def _pair(s, prec, monkeypatch, **kw):
    monkeypatch.setenv("RBMD_ONE_STREAM", "1")
    one, _ = make_ctx(s, prec, **kw)
    monkeypatch.delenv("RBMD_ONE_STREAM")
    two, _ = make_ctx(s, prec, **kw)
    for c in (one, two):
        c.set_state_u(s.u, vel=s.v, step=0)
    return one, two


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
@pytest.mark.parametrize("thermostat", [1, 3])
def test_two_streams_same_trajectory(sys5k, prec, thermostat, monkeypatch):
    import torch

    one, two = _pair(sys5k, prec, monkeypatch, rbe_P=120, seed=4, thermostat=thermostat,
                     temperature=1.0, tau_T=0.05, dt=0.002)
    for c in (one, two):
        c.step(2)
        c.step(4)  # replays the captured step graph
    u1, v1, s1 = one.get_state_u()
    u2, v2, s2 = two.get_state_u()
    assert s1 == s2 == 6
    assert torch.equal(u1, u2) and torch.equal(v1, v2)
    e1, e2 = one.energy(6), two.energy(6)
    for k in e1:
        assert np.array_equal(e1[k], e2[k]), k
    one.close()
    two.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_two_streams_energy_and_gradients(sys5k, prec, monkeypatch):
    import torch

    one, two = _pair(sys5k, prec, monkeypatch, rbe_P=120, seed=9)
    e1, e2 = one.energy(5), two.energy(5)
    for k in e1:
        assert np.array_equal(e1[k], e2[k]), k
    g1, g2 = one.energy_backward(5), two.energy_backward(5)
    for a, b in zip(g1, g2):
        if isinstance(a, torch.Tensor):
            assert torch.equal(a, b)
        else:
            assert np.array_equal(a, b)
    one.close()
    two.close()


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
def test_two_streams_forces_match_oracle(sys5k, prec, monkeypatch):
    import torch

    s = sys5k
    one, two = _pair(s, prec, monkeypatch, rbe_P=150, seed=7)
    F1 = one.forces(3)
    F2 = two.forces(3)
    assert torch.equal(F1, F2)
    Fo, _ = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 150, 7, 3)
    assert rel_err(to_np(F2), Fo) < TOL[prec]
    one.close()
    two.close()


def test_two_streams_batch(monkeypatch):
    import torch

    systems = synth.replicas([900, 2100, 333], seed=8, charges="1:1", n_types=2)
    cat = synth.concat(systems)
    dev = torch.device("cuda:0")

    def batch():
        b = rb.RBMD(torch.from_numpy(cat["x"]).to(dev), torch.from_numpy(cat["q"]).to(dev),
                    cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"], seed=[3, 4, 5],
                    replica=[0, 1, 2], rbe_P=60, thermostat=2, temperature=1.0, tau_T=0.1,
                    vel=torch.from_numpy(cat["v"]).to(dev))
        b.set_state_u(cat["u"], vel=cat["v"], step=0)
        return b

    monkeypatch.setenv("RBMD_ONE_STREAM", "1")
    one = batch()
    monkeypatch.delenv("RBMD_ONE_STREAM")
    two = batch()
    one.step(5)
    two.step(5)
    u1, v1, _ = one.get_state_u()
    u2, v2, _ = two.get_state_u()
    assert torch.equal(u1, u2) and torch.equal(v1, v2)
    one.close()
    two.close()


def test_rbe_only_and_rbl_only_stay_on_one_stream(sys5k):
    # with one part switched off there is nothing to overlap; the results are the
    # oracle's for the part that runs
    s = sys5k
    for flags, key in ((rb.NO_RBL, "rbe"), (rb.NO_RBE, "rbl")):
        ctx, _ = make_ctx(s, rb.FP64, rbe_P=80, seed=2, flags=flags)
        F = to_np(ctx.forces(1))
        if key == "rbe":
            Fo = to_np(ctx.rbe_forces(1))
        else:
            o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 2, 1)
            Fo = o["F"] - o["Fsum"] / s.n
        assert rel_err(F, Fo) < 1e-10, key
        ctx.close()


def test_user_stream(sys5k):
    # a context on a caller's stream: the fork and join of the force evaluation and
    # the host-buffer call order themselves against that stream, and the results
    # are those of a context on the default stream
    import torch

    s = sys5k
    ref, _ = make_ctx(s, rb.FP32, rbe_P=70, seed=9, thermostat=1)
    ref.set_state_u(s.u, vel=s.v, step=0)
    user = torch.cuda.Stream()
    with torch.cuda.stream(user):
        ctx, _ = make_ctx(s, rb.FP32, rbe_P=70, seed=9, thermostat=1)
        ctx.set_state_u(s.u, vel=s.v, step=0)
        assert ctx.stream.cuda_stream == user.cuda_stream
        ctx.step(3)
        F = ctx.forces(3)
        pos = torch.from_numpy(s.x).float().pin_memory()
        Fh = ctx.forces_host(pos, step=5)
    user.synchronize()
    ref.step(3)
    assert torch.equal(F, ref.forces(3))
    assert torch.equal(Fh, ref.forces_host(pos, step=5))
    ctx.close()
    ref.close()


def test_host_call_while_profiling(sys5k):
    # with stage events on (rbmd_profile) the host-buffer call runs its work in
    # sequence on one stream; the forces do not change
    import torch

    s = sys5k
    a, _ = make_ctx(s, rb.FP32, rbe_P=70, seed=10)
    b, _ = make_ctx(s, rb.FP32, rbe_P=70, seed=10)
    b.profile(True)
    pos = torch.from_numpy(s.x).float().pin_memory()
    assert torch.equal(a.forces_host(pos, step=2), b.forces_host(pos, step=2))
    a.close()
    b.close()
