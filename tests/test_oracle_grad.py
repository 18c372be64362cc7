"""Pins of the oracle's gradients of the total potential (charges, positions and
Lorentz-Berthelot LJ parameters).

  * every component equals a central finite difference of the oracle energy
    (list memberships held fixed: perturbations that would change a list are
    detected by comparing the lists and avoided);
  * with every shell member kept (exact lists) minus the position gradient is the
    force of orc_forces without the momentum correction; the RBE part of the
    position gradient is minus the RBE force (same draws);
  * the energies equal those of orc_forces.
"""
import numpy as np
import pytest

import oracle
from paper_2407_09315_b300 import synth

TWO32 = 2.0 ** 32


def _sys():
    return synth.electrolyte(120, seed=41, charges="2:1", n_types=3)


ARGS = dict(alpha=0.62, coulomb_k=1.3, r_core=2.0, r_cut=3.5, p=4, P=40, seed=5, step=2)


def _E(s, u=None, q=None, eps=None, sig=None, exact=False):
    E, *_ = oracle.energy_grad(s.u if u is None else u, s.q if q is None else q, s.types,
                               s.eps if eps is None else eps, s.sig if sig is None else sig,
                               s.L, exact=exact, **ARGS)
    return E.sum()


def _lists(s, u):
    o = oracle.rbl(u, s.q, s.types, s.eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                   ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["seed"], ARGS["step"])
    return o["n_core"], o["n_shell"], o["batch"]


def test_energies_match_forces_routine():
    s = _sys()
    E, *_ = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, **ARGS)
    _, Ef = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                          ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["P"], ARGS["seed"],
                          ARGS["step"])
    assert np.allclose(E, Ef, rtol=1e-12, atol=1e-12)


def test_position_gradient_by_finite_differences():
    s = _sys()
    _, dr, *_ = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, **ARGS)
    base = _lists(s, s.u)
    du = int(round(1e-6 * TWO32 / s.L))
    hx = du * s.L / TWO32
    checked = 0
    for i in range(0, s.n, 7):
        for d in range(3):
            up = s.u.copy(); dn = s.u.copy()
            up[i, d] = np.uint32((int(s.u[i, d]) + du) % 2 ** 32)
            dn[i, d] = np.uint32((int(s.u[i, d]) - du) % 2 ** 32)
            if any(not np.array_equal(a, b) for a, b in zip(_lists(s, up), base)) or \
               any(not np.array_equal(a, b) for a, b in zip(_lists(s, dn), base)):
                continue
            g = (_E(s, u=up) - _E(s, u=dn)) / (2 * hx)
            assert abs(g - dr[i, d]) <= 1e-4 * (abs(dr[i, d]) + 1e-3), (i, d, g, dr[i, d])
            checked += 1
    assert checked > 30


def test_charge_and_lj_gradients_by_finite_differences():
    s = _sys()
    _, _, dq, de, ds = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, **ARGS)
    h = 1e-6
    for i in (0, 17, 63, 119):
        qp = s.q.copy(); qm = s.q.copy()
        qp[i] += h; qm[i] -= h
        g = (_E(s, q=qp) - _E(s, q=qm)) / (2 * h)
        assert abs(g - dq[i]) <= 1e-4 * (abs(dq[i]) + 1e-3)
    for t in range(len(s.eps)):
        ep = s.eps.copy(); em = s.eps.copy()
        ep[t] += h; em[t] -= h
        g = (_E(s, eps=ep) - _E(s, eps=em)) / (2 * h)
        assert abs(g - de[t]) <= 1e-4 * (abs(de[t]) + 1e-3)
        sp = s.sig.copy(); sm = s.sig.copy()
        sp[t] += h; sm[t] -= h
        g = (_E(s, sig=sp) - _E(s, sig=sm)) / (2 * h)
        assert abs(g - ds[t]) <= 1e-4 * (abs(ds[t]) + 1e-3)


def test_exact_lists_give_minus_the_force():
    s = _sys()
    _, dr, *_ = oracle.energy_grad(s.u, s.q, s.types, s.eps, s.sig, s.L, exact=True, **ARGS)
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, ARGS["alpha"], ARGS["coulomb_k"],
                   ARGS["r_core"], ARGS["r_cut"], ARGS["p"], ARGS["seed"], ARGS["step"], exact=True)
    Fr, *_ = oracle.rbe_forces(s.u, s.q, s.L, ARGS["alpha"], ARGS["coulomb_k"], ARGS["P"],
                               ARGS["seed"], ARGS["step"])
    assert np.allclose(-dr, o["F"] + Fr, rtol=1e-10, atol=1e-10)
