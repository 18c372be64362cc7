"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2): the
job is N independent systems, one per rank (no data-path collective); the timing is
the slowest rank's and the throughput counts every rank's atoms."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, dev)
    sysr = bench.make_system(3000, 2 + rank, "c2")  # each rank its own seeded system
    h = float(np.sum(sysr.u.astype(np.float64)))
    hs = [None] * world
    dist.all_gather_object(hs, (sysr.n, h))
    dist.barrier()
    if rank == 0:
        out.put((t, hs))
    dist.destroy_process_group()


def test_two_rank_timing_and_weak_scaling():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, hs = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 15.0                      # the slowest rank's time
    assert hs[0][0] == hs[1][0] == 3000   # fixed work per rank (weak scaling)
    assert hs[0][1] != hs[1][1]           # independent systems
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(3000, 2, t) == pytest.approx(3000 * 2 / 0.015)
    assert bench.max_over_ranks(3.5, None, None) == 3.5
