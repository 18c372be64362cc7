"""rbmd_forces_host: host positions in, host forces out, with the copies
overlapping the kernels (chunks of structure-factor tiles).

The result must be bit for bit that of rbmd_set_state + rbmd_forces + a copy,
for one system and for a batch of replicas, in both precisions, with one chunk
(a system smaller than a tile) and several; the state afterwards is the same;
with one part of the method switched off the call runs the same work in
sequence.  One case is also checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import DEFAULTS, TOL, make_ctx, rel_err

pytestmark = pytest.mark.gpu


def _compare(ctx_ref, ctx_host, x, step, pinned=True):
    import torch

    dev = torch.device("cuda:0")
    pos_h = torch.from_numpy(x).to(ctx_ref.dtype)
    if pinned:
        pos_h = pos_h.pin_memory()
    ctx_ref.set_state(pos=pos_h.to(dev), step=step)
    F_ref = ctx_ref.forces(step).cpu()
    F_host = ctx_host.forces_host(pos_h, step=step)
    assert F_host.device.type == "cpu"
    assert torch.equal(F_host, F_ref)
    u1, _, s1 = ctx_ref.get_state_u()
    u2, _, s2 = ctx_host.get_state_u()
    assert s1 == s2 == step and torch.equal(u1, u2)
    return F_host


@pytest.mark.parametrize("prec", [rb.FP64, rb.FP32])
@pytest.mark.parametrize("n", [300, 5003])
def test_forces_host_equals_device_path(prec, n):
    s = synth.electrolyte(n, seed=41, charges="2:1", n_types=3)
    ref, _ = make_ctx(s, prec, rbe_P=90, seed=6)
    host, _ = make_ctx(s, prec, rbe_P=90, seed=6)
    for step in (0, 7):
        F = _compare(ref, host, s.x, step)
    if prec == rb.FP64 and n == 300:
        # the positions went through the encoder: the oracle runs at the encoded
        # fixed-point coordinates
        uu, _, _ = host.get_state_u()
        uu = (uu.cpu().numpy().astype(np.int64) % 2 ** 32).astype(np.uint32)
        Fo, _ = oracle.forces(uu, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 90, 6, 7)
        assert rel_err(F.numpy(), Fo) < TOL[rb.FP64]
    ref.close()
    host.close()


def test_forces_host_batch():
    import torch

    systems = synth.replicas([700, 2600, 4100], seed=9, charges="1:1", n_types=2)
    cat = synth.concat(systems)
    dev = torch.device("cuda:0")

    def batch():
        prm = dict(DEFAULTS)
        prm.update(rbe_P=70)
        return rb.RBMD(torch.from_numpy(cat["x"]).to(dev), torch.from_numpy(cat["q"]).to(dev),
                       cat["eps"], cat["sig"], box_length=cat["L"], n_atoms=cat["n"],
                       seed=[5, 6, 7], replica=[0, 1, 2], **prm)

    ref, host = batch(), batch()
    for step in (1, 4):
        _compare(ref, host, cat["x"], step)
    ref.close()
    host.close()


@pytest.mark.parametrize("flags", [rb.NO_RBE, rb.NO_RBL])
def test_forces_host_one_part(flags):
    s = synth.electrolyte(3000, seed=43, charges="2:1", n_types=3)
    ref, _ = make_ctx(s, rb.FP32, rbe_P=60, seed=3, flags=flags)
    host, _ = make_ctx(s, rb.FP32, rbe_P=60, seed=3, flags=flags)
    _compare(ref, host, s.x, 2)
    ref.close()
    host.close()


@pytest.mark.parametrize("chunks", [1, 3, 8])
def test_forces_host_pageable_and_chunks(chunks, monkeypatch):
    # pageable positions, and other chunk counts (RBMD_HOST_CHUNKS)
    s = synth.electrolyte(9000, seed=45, charges="2:1", n_types=2)
    ref, _ = make_ctx(s, rb.FP32, rbe_P=80, seed=8)
    host, _ = make_ctx(s, rb.FP32, rbe_P=80, seed=8)
    monkeypatch.setenv("RBMD_HOST_CHUNKS", str(chunks))
    _compare(ref, host, s.x, 3, pinned=False)
    _compare(ref, host, s.x, 4, pinned=True)
    ref.close()
    host.close()


def test_forces_host_rejects_device_tensors():
    import torch

    s = synth.electrolyte(300, seed=44, charges="1:1")
    ctx, _ = make_ctx(s, rb.FP32)
    with pytest.raises(ValueError):
        ctx.forces_host(torch.zeros((s.n, 3), device="cuda:0"))
    with pytest.raises(ValueError):
        ctx.forces_host(torch.zeros((s.n, 3), dtype=torch.float64))
    ctx.close()
