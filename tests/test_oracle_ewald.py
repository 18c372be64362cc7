"""Pins of the oracle's full Ewald sum (Sec. 2.2, Eqs. 5, 8, 10, 11).

  * rock-salt Madelung energy (tests/golden/madelung_nacl.txt) and zero forces
    by symmetry;
  * the total is independent of alpha at converged cutoffs, invariant under
    translation, and the forces sum to zero;
  * the conditionally convergent direct sum of Eq. 5, taken over spherical
    shells of images in a separate numpy loop, minus the surface (dipole) term
    converges to the tin-foil Ewald energy;
  * forces are minus the finite-difference gradients of the energies.
"""
import os

import numpy as np
import pytest

import oracle

TWO32 = 2.0 ** 32
GOLD = os.path.join(os.path.dirname(__file__), "golden", "madelung_nacl.txt")


def _madelung():
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            return float(line)


def _rocksalt(reps):
    """Rock salt with nearest-neighbour distance a = 1 in a box L = 2*reps."""
    L = 2.0 * reps
    g = np.arange(2 * reps)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    q = np.where(X.sum(1) % 2 == 0, 1.0, -1.0)
    u = (X * (TWO32 / L)).astype(np.uint64).astype(np.uint32)
    return u, q, L


def _total(e):
    return e["E_real"] + e["E_recip"] + e["E_self"]


@pytest.mark.parametrize("reps,alpha", [(1, 2.0), (4, 1.0)])
def test_madelung_rocksalt(reps, alpha):
    u, q, L = _rocksalt(reps)
    r_cut = 6.2 / np.sqrt(alpha)
    M = oracle.sampler_M(L, alpha)
    e = oracle.ewald(u, q, L, alpha, 1.0, r_cut, M)
    E_per_ion = _total(e) / len(q)
    assert abs(E_per_ion - (-_madelung() / 2.0)) < 1e-6
    F = e["F_real"] + e["F_recip"]
    assert np.max(np.abs(F)) < 1e-12


def _random_neutral(n, L, seed):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2 ** 32, size=(n, 3), dtype=np.uint64).astype(np.uint32)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q[:4] *= 2.0  # mixed valences, still neutral
    return u, q


def test_alpha_independence_and_invariants():
    n, L = 64, 6.84
    u, q = _random_neutral(n, L, 5)
    # keep atoms apart so that the energy is well conditioned
    tot = []
    for alpha in (0.3, 0.62, 1.2):
        e = oracle.ewald(u, q, L, alpha, 1.0, 6.2 / np.sqrt(alpha), oracle.sampler_M(L, alpha))
        tot.append(_total(e))
        F = e["F_real"] + e["F_recip"]
        assert np.linalg.norm(F.sum(0)) < 1e-12 * np.abs(F).sum()
        # the Fourier part alone sums to zero too
        assert np.linalg.norm(e["F_recip"].sum(0)) < 1e-12 * np.abs(e["F_recip"]).sum()
    tot = np.array(tot)
    assert np.max(np.abs(tot - tot[1])) < 1e-9 * abs(tot[1])
    # rigid translation (exact in fixed point)
    shift = np.array([123456789, 987654321, 55555], dtype=np.uint64)
    u2 = ((u.astype(np.uint64) + shift) % 2 ** 32).astype(np.uint32)
    alpha = 0.62
    e1 = oracle.ewald(u, q, L, alpha, 1.0, 6.2 / np.sqrt(alpha), oracle.sampler_M(L, alpha))
    e2 = oracle.ewald(u2, q, L, alpha, 1.0, 6.2 / np.sqrt(alpha), oracle.sampler_M(L, alpha))
    assert abs(_total(e1) - _total(e2)) < 1e-11 * abs(_total(e1))
    assert np.allclose(e1["F_real"] + e1["F_recip"], e2["F_real"] + e2["F_recip"],
                       rtol=1e-9, atol=1e-10)


def _sphere_sum(x, q, L, R):
    """Eq. 5 summed over image cells with |n| <= R (spherical order)."""
    r = np.arange(-R, R + 1)
    n3 = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    n3 = n3[(n3 ** 2).sum(1) <= R * R]
    E = 0.0
    for i in range(len(q)):
        for j in range(len(q)):
            d = x[i] - x[j] + n3 * L
            rr = np.sqrt((d * d).sum(1))
            if i == j:
                rr = rr[rr > 0]
            E += 0.5 * q[i] * q[j] * np.sum(1.0 / rr)
    return E


def test_direct_image_sum_converges_to_ewald():
    rng = np.random.default_rng(3)
    L = 1.0
    u = rng.integers(0, 2 ** 32, size=(4, 3), dtype=np.uint64).astype(np.uint32)
    q = np.array([1.0, -1.0, 2.0, -2.0])
    x = u.astype(float) * (L / TWO32)
    alpha = 30.0
    e = oracle.ewald(u, q, L, alpha, 1.0, 6.2 / np.sqrt(alpha), oracle.sampler_M(L, alpha))
    D = (q[:, None] * x).sum(0)
    surface = 2.0 * np.pi * np.dot(D, D) / (3.0 * L ** 3)
    errs = [abs(_sphere_sum(x, q, L, R) - surface - _total(e)) for R in (10, 20, 30)]
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 1e-6 * abs(_total(e))
    # without the surface term the spherical sum is a different (vacuum) energy
    assert abs(_sphere_sum(x, q, L, 30) - _total(e)) > 0.1


def test_real_space_part_is_an_explicit_image_sum():
    # erfc part of Eq. 8 by a plain numpy loop over images within r_cut
    from scipy.special import erfc
    rng = np.random.default_rng(9)
    n, L, alpha, r_cut = 12, 5.0, 0.8, 4.0
    u, q = _random_neutral(n, L, 9)
    x = u.astype(float) * (L / TWO32)
    E = 0.0
    r = np.arange(-2, 3)
    n3 = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    for i in range(n):
        for j in range(n):
            d = x[i] - x[j] + n3 * L
            rr = np.sqrt((d * d).sum(1))
            keep = (rr < r_cut) & (rr > 0)
            E += 0.5 * q[i] * q[j] * np.sum(erfc(np.sqrt(alpha) * rr[keep]) / rr[keep])
    e = oracle.ewald(u, q, L, alpha, 1.0, r_cut, 2)
    assert abs(e["E_real"] - E) < 1e-12 * abs(E)


def _fd_check(energy_fn, force, u, L, atoms, h=1e-5, tol=1e-6):
    du = int(round(h * TWO32 / L))
    hx = du * L / TWO32
    for i in atoms:
        for d in range(3):
            up = u.copy(); dn = u.copy()
            up[i, d] = np.uint32((int(u[i, d]) + du) % 2 ** 32)
            dn[i, d] = np.uint32((int(u[i, d]) - du) % 2 ** 32)
            g = (energy_fn(up) - energy_fn(dn)) / (2 * hx)
            assert abs(-g - force[i, d]) <= tol * (abs(force[i, d]) + 1.0), (i, d, -g, force[i, d])


def test_ewald_forces_are_energy_gradients():
    n, L, alpha = 16, 5.0, 1.0
    u, q = _random_neutral(n, L, 21)
    r_cut = 6.2 / np.sqrt(alpha)
    M = oracle.sampler_M(L, alpha)
    e = oracle.ewald(u, q, L, alpha, 1.0, r_cut, M)
    _fd_check(lambda uu: oracle.ewald(uu, q, L, alpha, 1.0, r_cut, M)["E_recip"],
              e["F_recip"], u, L, atoms=[0, 5, 11])
    _fd_check(lambda uu: oracle.ewald(uu, q, L, alpha, 1.0, r_cut, M)["E_real"],
              e["F_real"], u, L, atoms=[1, 7])


def test_coulomb_prefactor_scales_linearly():
    n, L, alpha = 8, 4.0, 1.5
    u, q = _random_neutral(n, L, 2)
    r_cut = 6.2 / np.sqrt(alpha)
    M = oracle.sampler_M(L, alpha)
    e1 = oracle.ewald(u, q, L, alpha, 1.0, r_cut, M)
    e2 = oracle.ewald(u, q, L, alpha, 3.5, r_cut, M)
    assert abs(_total(e2) - 3.5 * _total(e1)) < 1e-12 * abs(_total(e2))
