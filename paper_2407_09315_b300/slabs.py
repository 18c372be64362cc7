"""Spatial decomposition of one system over several GPUs (slabs along x).

The paper names parallel GPUs as future work (Sec. 5).  The split follows the
method's structure: the RBE structure factors (Eq. 9) are sums over atoms, so each
rank sums the atoms it owns and the ranks exchange 2P numbers per step; the RBL
(Sec. 2.3) needs, for an owned atom, only the atoms within r_cut, so each rank
also holds a halo of the other ranks' atoms near its slab.

This module holds the host-side bookkeeping (which atoms a rank owns and which
halo atoms it needs, decided on the integer fixed-point coordinates) and the
order of the exchanges; every force is computed by the CUDA library's slab
contexts (rbmd_init_slab and its calls):

  1. every rank: exact partial structure factors of its owned atoms;
  2. exchange: every rank adds all ranks' sums in rank order (integers: the
     result does not depend on the order, and with atom tiles that hold the same
     atoms it is bit for bit that of one context holding every atom);
  3. every rank: RBL forces of its owned atoms and their sum;
  4. exchange: the sums, added in rank order, give the momentum correction;
  5. every rank: correction added, RBE forces from the summed structure factors.

The exchanges are two all-gathers (4P int64 and 3 doubles per rank); with
torch.distributed they run on whichever backend the process group uses.
"""
from __future__ import annotations

import math

import numpy as np

TWO32 = 1 << 32


def slab_bounds(n_ranks):
    """Equal x-slabs: rank r owns 0 <= u_x < 2^32 with floor(u_x n / 2^32) == r,
    i.e. u_x in [ceil(r 2^32/n), ceil((r+1) 2^32/n))."""
    return [-(-r * TWO32 // n_ranks) for r in range(n_ranks + 1)]


def halo_margin(r_cut, box_length):
    """Largest |dx| (fixed-point units) of a pair the library can count as a
    neighbour: sqrt(floor((r_cut 2^32/L)^2)) rounded down, plus one unit."""
    s = r_cut * (TWO32 / box_length)
    return math.isqrt(int(math.floor(s * s))) + 1


def slab_partition(u, box_length, n_ranks, r_cut, bounds=None):
    """Owned and halo atom ids (numpy int64 arrays, ascending) of every rank.

    u: uint32 [N, 3] fixed-point coordinates of the whole system.  bounds: n+1
    increasing x boundaries in fixed-point units, bounds[0] = 0 and bounds[n] = 2^32
    (default: equal slabs).  A rank's halo holds every atom of the other ranks
    whose periodic x-distance to the rank's slab is at most halo_margin: all atoms
    within r_cut of an owned atom are there (the distance along x of such a pair
    is at most the margin)."""
    if bounds is None:
        bounds = slab_bounds(n_ranks)
    if len(bounds) != n_ranks + 1 or bounds[0] != 0 or bounds[-1] != TWO32:
        raise ValueError("bounds must run from 0 to 2^32 with one slab per rank")
    ux = np.asarray(u)[:, 0].astype(np.int64)
    owner = np.searchsorted(np.asarray(bounds[1:-1], dtype=np.int64), ux, side="right")
    m = halo_margin(r_cut, box_length)
    owned, halo = [], []
    for r in range(n_ranks):
        lo, hi = bounds[r], bounds[r + 1] - 1
        if hi < lo:
            raise ValueError("empty slab")
        # periodic distance of x to the interval [lo, hi]
        below = (lo - ux) % TWO32
        above = (ux - hi) % TWO32
        inside = (ux >= lo) & (ux <= hi)
        dist = np.where(inside, 0, np.minimum(below, above))
        own = np.nonzero(owner == r)[0]
        hal = np.nonzero((owner != r) & (dist <= m))[0]
        owned.append(own.astype(np.int64))
        halo.append(hal.astype(np.int64))
    return owned, halo


def _gather_dist(value):
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(value))
    if dist.get_backend() == "nccl":
        t = t.cuda()
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return [o.cpu().numpy() for o in out]


class SlabRank:
    """One rank's slab context: the owned atoms of `owned` (global ids) followed by
    the halo atoms, with the global box and parameters.  `params` are those of
    paper_2407_09315_b300.RBMD (alpha, r_core, r_cut, rbl_p, rbe_P, seed, ...)."""

    def __init__(self, u, q, types, eps, sig, box_length, owned, halo, *, precision,
                 device, **params):
        import torch

        import paper_2407_09315_b300 as rb

        self.owned = np.asarray(owned, dtype=np.int64)
        self.halo = np.asarray(halo, dtype=np.int64)
        rows = np.concatenate([self.owned, self.halo])
        self.rows = rows
        n_global = len(q)
        dt = torch.float64 if precision == rb.FP64 else torch.float32
        uu = np.ascontiguousarray(np.asarray(u)[rows], dtype=np.uint32)
        x = uu.astype(np.float64) * (box_length / TWO32)
        self.ctx = rb.RBMD(torch.from_numpy(x).to(device, dt),
                           torch.from_numpy(np.asarray(q)[rows]).to(device, dt), eps, sig,
                           box_length=box_length, precision=precision,
                           types=torch.from_numpy(np.asarray(types)[rows].astype(np.int32)).to(device),
                           slab=(len(self.owned), n_global,
                                 torch.from_numpy(rows.astype(np.int32))), **params)
        self.ctx.set_state_u(uu, step=0)
        self.n_owned = len(self.owned)

    def close(self):
        self.ctx.close()


def slab_forces_local(ranks, step):
    """Forces of all atoms from the slab contexts of every rank in this process
    (the exchanges done in memory, in rank order).  Returns the [N, 3] numpy array
    in global atom order, and the summed structure factors."""
    import paper_2407_09315_b300 as rb

    accs = [r.ctx.rho_partial(step) for r in ranks]
    total = np.zeros_like(accs[0])
    for a in accs:
        rb.rho_acc_add(total, a)
    forces, fsums = [], []
    for r in ranks:
        F, fs = r.ctx.rbl_forces_slab(step)
        forces.append(F)
        fsums.append(fs)
    fsum = np.zeros(3)
    for fs in fsums:
        fsum = fsum + fs
    n_global = sum(r.n_owned for r in ranks)
    out = np.zeros((n_global, 3))
    for r, F in zip(ranks, forces):
        r.ctx.add_correction(F, fsum)
        r.ctx.forces_rho(step, total, out=F, accumulate=True)
        out[r.owned] = F[:r.n_owned].double().cpu().numpy()
    return out, total


def slab_forces_dist(rank, step):
    """Forces of this rank's owned atoms (torch tensor [n_owned, 3]) with the two
    exchanges as torch.distributed all-gathers (every rank calls it)."""
    import paper_2407_09315_b300 as rb

    acc = rank.ctx.rho_partial(step)
    total = np.zeros_like(acc)
    for a in _gather_dist(acc):
        rb.rho_acc_add(total, a)
    F, fs = rank.ctx.rbl_forces_slab(step)
    fsum = np.zeros(3)
    for f in _gather_dist(fs):
        fsum = fsum + f
    rank.ctx.add_correction(F, fsum)
    rank.ctx.forces_rho(step, total, out=F, accumulate=True)
    return F[:rank.n_owned]
