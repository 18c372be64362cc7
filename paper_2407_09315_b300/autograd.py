"""torch.autograd.Function over the potential energy of one step.

E(pos, q, eps, sigma) = E_coul_real + E_lj + E_rbe + E_self with the random draws
(RBE modes and RBL batches) of `step` held fixed.  Forward calls rbmd_energy,
backward calls rbmd_energy_backward (hand-written adjoint kernels); the
structure factors are recomputed on the backward pass, never stored per atom.
"""
from __future__ import annotations

import numpy as np
import torch


class Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, step, pos, q, eps, sigma):
        sim.set_state(pos=pos.detach().to(sim.device, sim.dtype).contiguous(), step=step)
        sim.set_charges(q.detach())
        sim.set_lj(eps.detach().cpu().double().numpy(), sigma.detach().cpu().double().numpy())
        e = sim.energy(step)["e_potential"]
        ctx.sim = sim
        ctx.step = step
        ctx.meta = (pos.dtype, pos.device, q.dtype, eps.dtype, eps.device)
        return torch.tensor(e, dtype=torch.float64, device=pos.device)

    @staticmethod
    def backward(ctx, grad_out):
        sim = ctx.sim
        pdt, pdev, qdt, edt, edev = ctx.meta
        g = float(grad_out.detach().cpu())
        dpos, dq, de, ds = sim.energy_backward(ctx.step, g, want_pos=ctx.needs_input_grad[2],
                                              want_q=ctx.needs_input_grad[3],
                                              want_lj=ctx.needs_input_grad[4] or
                                              ctx.needs_input_grad[5])
        out_pos = dpos.to(pdev, pdt) if dpos is not None else None
        out_q = dq.to(pdev, qdt) if dq is not None else None
        out_e = torch.from_numpy(np.asarray(de)).to(edev, edt) if de is not None else None
        out_s = torch.from_numpy(np.asarray(ds)).to(edev, edt) if ds is not None else None
        return None, None, out_pos, out_q, out_e, out_s


def energy(sim, step, pos, q, eps, sigma):
    """Differentiable potential energy of `sim` at `step` (see Energy)."""
    return Energy.apply(sim, step, pos, q, eps, sigma)
