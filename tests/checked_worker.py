"""Runs a set of library calls and saves their results (npz), for the comparison
of the bounds-checked build with the default one (tests/test_gpu_checked.py runs
it once per library, each in a process of its own)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))


def main(out_path):
    import paper_2407_09315_b300 as rb
    from paper_2407_09315_b300 import slabs, synth
    from gpu_util import make_ctx, to_np
    import torch

    res = {}
    s = synth.electrolyte(3001, seed=121, charges="2:1", n_types=3)
    for prec, tag in ((rb.FP32, "f32"), (rb.FP64, "f64")):
        ctx, _ = make_ctx(s, prec, seed=4, thermostat=1)
        res[tag + "_forces"] = to_np(ctx.forces(2))
        nc, ns, b = (to_np(t) for t in ctx.rbl_lists(2))
        res[tag + "_lists"] = np.concatenate([nc[:, None], ns[:, None], b], axis=1)
        ctx.set_state_u(s.u, vel=s.v, step=0)
        ctx.step(5)  # the candidate lists, their rebuilds and the step graph
        u, v, _ = ctx.get_state_u()
        res[tag + "_u"] = to_np(u)
        res[tag + "_v"] = to_np(v)
        E = ctx.energy(5)
        res[tag + "_e"] = np.array([E["e_coul_real"], E["e_lj"], E["e_rbe"]])
        dpos, dq, de, ds = ctx.energy_backward(5)
        res[tag + "_grad"] = np.concatenate([to_np(dpos).ravel(), to_np(dq), de, ds])
        ctx.close()
    # overflow fallback and slab contexts
    os.environ["RBMD_LIST_CAPS"] = "4,12"
    ctx, _ = make_ctx(s, rb.FP32, seed=4)
    del os.environ["RBMD_LIST_CAPS"]
    res["ovf_forces"] = to_np(ctx.forces(1))
    ctx.close()
    owned, halo = slabs.slab_partition(s.u, s.L, 2, 3.5)
    ranks = [slabs.SlabRank(s.u, s.q, s.types, s.eps, s.sig, s.L, owned[r], halo[r],
                            precision=rb.FP32, device=torch.device("cuda:0"), seed=4, rbe_P=100)
             for r in range(2)]
    res["slab_forces"], _ = slabs.slab_forces_local(ranks, 1)
    for r in ranks:
        r.close()
    torch.cuda.synchronize()
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
