"""Seeded synthetic electrolytes: the inputs of every test and benchmark.

This module only makes inputs (positions, charges, LJ types and parameters,
velocities).  It holds none of the method's arithmetic, so both the CUDA
library and the FP64 oracle can be fed from it.

Recipe (reduced units, cubic periodic box, number density 0.2 per sigma^3):
  * positions uniform in the box, then every pair closer than
    d_min(i, j) = dmin_factor * sigma_ij is resolved by redrawing the
    higher-index atom until no pair is left (a uniform hard-core fluid at a
    packing fraction of about 5 %);
  * charges: "1:1" gives +1/-1 by index parity; "2:1" gives floor(N/3)
    cations +2, 2*floor(N/3) anions -1 and the rest neutral, so the total
    charge is exactly zero; the charges are shuffled over the atoms;
  * LJ types uniform per atom; per-type sigma ~ U[sigma_lo, sigma_hi] and
    epsilon ~ U[eps_lo, eps_hi] (a single type gets sigma = epsilon = 1);
  * velocities Maxwell-Boltzmann at T0 with unit masses, centre-of-mass
    motion removed and rescaled so that 2 KE / (3N - 3) = T0 exactly.
Randomness is numpy's PCG64 seeded with ``seed``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

TWO32 = 4294967296.0


@dataclasses.dataclass
class System:
    L: float
    u: np.ndarray          # uint32 [N, 3] fixed-point fractional coordinates
    q: np.ndarray          # float64 [N]
    types: np.ndarray      # int32 [N]
    eps: np.ndarray        # float64 [T]
    sig: np.ndarray        # float64 [T]
    v: np.ndarray          # float64 [N, 3]

    @property
    def n(self) -> int:
        return len(self.q)

    @property
    def x(self) -> np.ndarray:
        return self.u.astype(np.float64) * (self.L / TWO32)


def box_length(n: int, density: float = 0.2) -> float:
    return float((n / density) ** (1.0 / 3.0))


def _place(n, L, types, sig, dmin_factor, rng, max_iter=500):
    from scipy.spatial import cKDTree

    x = rng.uniform(0.0, L, size=(n, 3))
    if n < 2 or dmin_factor <= 0:
        return x
    dmax = dmin_factor * float(np.max(sig))
    check = None  # atoms whose neighbourhoods must be checked (None: all)
    for _ in range(max_iter):
        x = np.mod(x, L)
        x[x >= L] = 0.0
        tree = cKDTree(x, boxsize=L)
        if check is None:
            pairs = tree.query_pairs(dmax, output_type="ndarray")
        else:
            nb = tree.query_ball_point(x[check], dmax)
            cnt = np.fromiter((len(a) for a in nb), dtype=np.int64, count=len(nb))
            if cnt.sum() == 0:
                return x
            j = np.concatenate([np.asarray(a, dtype=np.int64) for a in nb])
            i = np.repeat(check, cnt)
            keep = i != j
            pairs = np.stack([i[keep], j[keep]], axis=1)
        if len(pairs) == 0:
            return x
        d = x[pairs[:, 0]] - x[pairs[:, 1]]
        d -= L * np.round(d / L)
        r = np.sqrt(np.sum(d * d, axis=1))
        sij = 0.5 * (sig[types[pairs[:, 0]]] + sig[types[pairs[:, 1]]])
        bad = r < dmin_factor * sij
        if not np.any(bad):
            return x
        redo = np.unique(np.maximum(pairs[bad, 0], pairs[bad, 1]))
        x[redo] = rng.uniform(0.0, L, size=(len(redo), 3))
        check = redo
    raise RuntimeError("hard-core placement did not converge")


def to_fixed(x: np.ndarray, L: float) -> np.ndarray:
    f = np.floor(np.mod(x, L) * (TWO32 / L))
    f = np.clip(f, 0, TWO32 - 1)
    return f.astype(np.uint64).astype(np.uint32)


def maxwell_boltzmann(n: int, T0: float, rng) -> np.ndarray:
    v = rng.normal(0.0, np.sqrt(T0), size=(n, 3))
    if n > 1:
        v -= v.mean(axis=0)
        ke = 0.5 * np.sum(v * v)
        T = 2.0 * ke / (3.0 * n - 3.0)
        if T > 0:
            v *= np.sqrt(T0 / T)
    return v


def electrolyte(n: int, L: float | None = None, density: float = 0.2, seed: int = 0,
                charges: str = "1:1", n_types: int = 1, sigma_range=(0.8, 1.2),
                eps_range=(0.5, 1.5), dmin_factor: float = 0.8, T0: float = 1.0,
                lj=None) -> System:
    """lj: optional (eps, sigma) per type to use instead of drawing them."""
    rng = np.random.default_rng(seed)
    if L is None:
        L = box_length(n, density)
    if lj is not None:
        eps = np.asarray(lj[0], dtype=np.float64)
        sig = np.asarray(lj[1], dtype=np.float64)
        n_types = len(eps)
    elif n_types == 1:
        sig = np.ones(1)
        eps = np.ones(1)
    else:
        sig = rng.uniform(sigma_range[0], sigma_range[1], size=n_types)
        eps = rng.uniform(eps_range[0], eps_range[1], size=n_types)
    types = rng.integers(0, n_types, size=n).astype(np.int32)
    if charges == "1:1":
        q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
        if n % 2 == 1:
            q[-1] = 0.0
    elif charges == "2:1":
        nc = n // 3
        q = np.zeros(n)
        q[:nc] = 2.0
        q[nc:3 * nc] = -1.0
        q = q[rng.permutation(n)]
    else:
        raise ValueError(charges)
    x = _place(n, L, types, sig, dmin_factor, rng)
    u = to_fixed(x, L)
    v = maxwell_boltzmann(n, T0, rng)
    return System(L=float(L), u=u, q=q.astype(np.float64), types=types, eps=eps, sig=sig, v=v)


# Workloads of the benchmark and the parity tests (sizes, charges, types).
def config1() -> System:
    """N=1000 monovalent ions (500 +1, 500 -1), L=17.1, one LJ type, seed 0."""
    return electrolyte(1000, L=17.1, seed=0, charges="1:1", n_types=1)


def config2() -> System:
    """N=100,000 monovalent ions at density 0.2, seed 1."""
    return electrolyte(100_000, seed=1, charges="1:1", n_types=1)


def config3() -> System:
    """N=1,000,000 2:1 electrolyte, 4 LJ types, density 0.2, seed 2."""
    return electrolyte(1_000_000, seed=2, charges="2:1", n_types=4)


def config4() -> System:
    """N=10,000,000 monovalent ions at density 0.2, seed 3."""
    return electrolyte(10_000_000, seed=3, charges="1:1", n_types=1)


def replica_sizes(n_rep: int = 64, lo: int = 2000, hi: int = 200_000, seed: int = 4):
    """Even N_r drawn log-uniformly in [lo, hi] (batched workload)."""
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_rep))
    return (2 * np.round(x / 2)).astype(np.int64)


def replicas(sizes, seed: int = 4, density: float = 0.2, charges: str = "1:1",
             n_types: int = 1, T0=1.0) -> list:
    """Independent systems of the given sizes sharing one set of LJ parameters
    (drawn from ``seed``); replica r is seeded with 1000 * seed + r + 1.  T0 may
    be a scalar or one temperature per replica."""
    base = electrolyte(max(int(n_types), 2) if n_types > 1 else 2, seed=seed, n_types=n_types,
                       charges="1:1", dmin_factor=0.0)
    T0s = list(T0) if np.ndim(T0) > 0 else [T0] * len(sizes)
    return [electrolyte(int(n), density=density, seed=1000 * seed + r + 1, charges=charges,
                        lj=(base.eps, base.sig), T0=T0s[r])
            for r, n in enumerate(sizes)]


def concat(systems) -> dict:
    """The concatenated arrays of a batch of systems (replica order)."""
    return dict(u=np.concatenate([s.u for s in systems]),
                x=np.concatenate([s.x for s in systems]),
                q=np.concatenate([s.q for s in systems]),
                types=np.concatenate([s.types for s in systems]),
                v=np.concatenate([s.v for s in systems]),
                L=[s.L for s in systems], n=[s.n for s in systems],
                eps=systems[0].eps, sig=systems[0].sig)
