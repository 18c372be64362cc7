"""Shared helpers of the GPU parity tests: build a context from a synthetic
system with exact fixed-point positions, and the error norms used everywhere.

Tolerances (force RMS relative error ||F - F_ref||_2 / ||F_ref||_2 against the
FP64 oracle): 1e-5 for the FP32 path, 1e-10 for the FP64 path; integer results
(modes, list counts, batches) must match exactly.
"""
import numpy as np

import paper_2407_09315_b300 as rb

TOL = {rb.FP32: 1e-5, rb.FP64: 1e-10}
DEFAULTS = dict(alpha=0.62, r_core=2.0, r_cut=3.5, rbl_p=10, rbe_P=100, coulomb_k=1.0)


def make_ctx(system, precision=rb.FP64, **kw):
    import torch

    dt = torch.float64 if precision == rb.FP64 else torch.float32
    prm = dict(DEFAULTS)
    prm.update(kw)
    dev = torch.device("cuda:0")
    pos = torch.from_numpy(system.x).to(dev, dt)
    q = torch.from_numpy(system.q).to(dev, dt)
    vel = torch.from_numpy(system.v).to(dev, dt)
    types = torch.from_numpy(system.types).to(dev)
    ctx = rb.RBMD(pos, q, system.eps, system.sig, box_length=system.L, precision=precision,
                  vel=vel, types=types, **prm)
    ctx.set_state_u(system.u, step=0)
    return ctx, prm


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)
