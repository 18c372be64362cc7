"""The allocation-free RBE force entry point (rbmd_rbe_forces_noalloc).

Some callers cannot allocate device memory (another framework owns the device
memory pool, or an allocation would synchronise a latency-critical path).  The
entry point serves them with a fixed static scratch array.  Its output must
match the FP64 oracle's RBE force (Eq. 12) and the context entry point
rbmd_rbe_forces within the FP32 tolerance of the other parity tests, on two
calls in a row (the second reuses the scratch the first one left behind).  P
runs up to the static maximum (each structure-factor thread owns modes l and
l + 256, so P = 300 and 512 take the second half of the mode range).  This file
is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import TOL, make_ctx, rel_err, to_np


@pytest.mark.gpu
@pytest.mark.parametrize("P", [200, 300, 512])
def test_noalloc_matches_oracle_and_context_twice(P):
    import torch

    s = synth.electrolyte(5003, seed=31, charges="2:1", n_types=2)
    ctx, _ = make_ctx(s, rb.FP32, rbe_P=P, seed=7, replica=2)
    dev = torch.device("cuda:0")
    u = torch.from_numpy(np.ascontiguousarray(s.u).view(np.int32)).to(dev)
    q = torch.from_numpy(s.q).to(dev, torch.float32)
    out = torch.full((s.n, 3), float("nan"), dtype=torch.float32, device=dev)
    for step in (3, 4):
        Fo, _, _, _ = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, P, 7, step, replica=2)
        ref = to_np(ctx.rbe_forces(step))
        rb.rbe_forces_noalloc(u, q, s.L, alpha=0.62, coulomb_k=1.0, P=P, seed=7, step=step,
                              replica=2, out=out)
        torch.cuda.synchronize()
        got = to_np(out)
        assert np.all(np.isfinite(got))
        assert rel_err(got, Fo) < TOL[rb.FP32], (P, step, rel_err(got, Fo))
        assert rel_err(got, ref) < TOL[rb.FP32], (P, step, rel_err(got, ref))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = rb.lib()
    dummy = np.zeros(16, dtype=np.float32)
    p = dummy.ctypes.data_as(C.c_void_p)
    # P above the static maximum: rejected before any device work
    assert lib.rbmd_rbe_forces_noalloc(p, p, 4, 10.0, 0.6, 1.0, 513, 0, 0, 0, p, None) == 1
    # box so large for alpha that the sampler table would not fit
    assert lib.rbmd_rbe_forces_noalloc(p, p, 4, 1.0e5, 0.6, 1.0, 16, 0, 0, 0, p, None) == 1
    assert lib.rbmd_rbe_forces_noalloc(None, p, 4, 10.0, 0.6, 1.0, 16, 0, 0, 0, p, None) == 1


def test_noalloc_wrapper_rejects_bad_tensors():
    # the binding checks device, dtype, shape and contiguity before any call
    import torch

    u = torch.zeros((4, 3), dtype=torch.int32)
    q = torch.zeros(4, dtype=torch.float32)
    out = torch.zeros((4, 3), dtype=torch.float32)
    with pytest.raises(ValueError):
        rb.rbe_forces_noalloc(u, q, 10.0, alpha=0.6, coulomb_k=1.0, P=8, seed=0, step=0,
                              out=out)
