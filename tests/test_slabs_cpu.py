"""Host-side bookkeeping of the spatial decomposition (paper_2407_09315_b300.slabs),
on the CPU: the slab partition and its halos, and the two exchanges of a
distributed force evaluation run as world-size-2 gloo ranks.

  * every atom is owned by exactly one rank; a rank's halo holds no owned atom;
  * every atom within r_cut of an owned atom (minimum image) is owned or in the
    halo, for equal slabs, uneven boundaries and slabs thinner than r_cut;
  * the exact structure-factor sums (128-bit words) gathered over gloo and added
    in rank order give every rank the same total, equal to the direct integer sum,
    and the force sums for the momentum correction agree on every rank.
"""
import os

import numpy as np
import pytest

import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import slabs, synth


def _neighbours_present(s, r_cut, owned, halo):
    x = s.x
    have = np.zeros(s.n, dtype=bool)
    have[owned] = True
    have[halo] = True
    for i in owned[:: max(1, len(owned) // 300)]:
        d = x - x[i]
        d -= s.L * np.round(d / s.L)
        near = np.nonzero((d * d).sum(1) <= r_cut * r_cut * (1 + 1e-9))[0]
        assert have[near].all(), (i, near[~have[near]])


@pytest.mark.parametrize("n_ranks,bounds", [(2, None), (3, None), (4, "uneven")])
def test_partition_owns_once_and_halos_are_complete(n_ranks, bounds):
    s = synth.electrolyte(6000, seed=101, charges="1:1", n_types=1)
    if bounds == "uneven":
        q = np.sort(s.u[:, 0].astype(np.int64))
        bounds = [0, int(q[1000]), int(q[1024 * 3]), int(q[5000]), 1 << 32]
    owned, halo = slabs.slab_partition(s.u, s.L, n_ranks, 3.5, bounds=bounds)
    cnt = np.zeros(s.n, dtype=int)
    for o in owned:
        cnt[o] += 1
    assert np.all(cnt == 1)
    for r in range(n_ranks):
        assert not np.intersect1d(owned[r], halo[r]).size
        _neighbours_present(s, 3.5, owned[r], halo[r])


def test_thin_slabs_still_complete():
    # 8 slabs of width L/8 < r_cut: the halo reaches across several slabs
    s = synth.electrolyte(2000, seed=102, charges="1:1", n_types=1)
    assert s.L / 8 < 3.5
    owned, halo = slabs.slab_partition(s.u, s.L, 8, 3.5)
    for r in range(8):
        _neighbours_present(s, 3.5, owned[r], halo[r])


def test_rho_acc_add_is_exact_128_bit():
    rng = np.random.default_rng(5)
    parts = [rng.integers(-2 ** 62, 2 ** 62, size=(7, 4), dtype=np.int64) for _ in range(5)]
    for p in parts:  # low words are unsigned halves: any bit pattern
        p[:, 0] = rng.integers(-2 ** 63, 2 ** 63 - 1, size=7, dtype=np.int64)
        p[:, 2] = rng.integers(-2 ** 63, 2 ** 63 - 1, size=7, dtype=np.int64)
    tot = np.zeros((7, 4), dtype=np.int64)
    for p in parts:
        rb.rho_acc_add(tot, p)

    def val(a, k, c):
        return (int(a[k, 2 * c + 1]) << 64) + (int(a[k, 2 * c]) & ((1 << 64) - 1))

    for k in range(7):
        for c in range(2):
            want = sum(val(p, k, c) for p in parts)
            want = (want + (1 << 127)) % (1 << 128) - (1 << 127)
            assert val(tot, k, c) == want


def _exchange_rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(100 + rank)
        acc = rng.integers(-2 ** 40, 2 ** 40, size=(9, 4), dtype=np.int64)
        fs = rng.standard_normal(3)
        total = np.zeros_like(acc)
        for a in slabs._gather_dist(acc):
            rb.rho_acc_add(total, a)
        fsum = np.zeros(3)
        for f in slabs._gather_dist(fs):
            fsum = fsum + f
        q.put((rank, acc, fs, total, fsum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_exchanges():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_exchange_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(2)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    direct = np.zeros_like(res[0][1])
    rb.rho_acc_add(direct, res[0][1])
    rb.rho_acc_add(direct, res[1][1])
    for _, _, _, total, fsum in res:
        assert np.array_equal(total, direct)
        assert np.array_equal(fsum, res[0][4])
    assert np.array_equal(res[0][4], res[0][2] + res[1][2])
