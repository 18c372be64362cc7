"""The oracle's host threads (the CPU baseline's all-cores leg) change no
per-atom result: every force component is computed by the same operations in
the same order for any thread count; only the order of the sums over atoms
(F_corr, energies, virials) changes, within rounding."""
import numpy as np

import oracle
from paper_2407_09315_b300 import synth


def test_threads_give_the_same_forces():
    s = synth.electrolyte(3000, seed=81, charges="2:1", n_types=2)
    args = (s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 7, 3)
    oracle.set_threads(1)
    o1 = oracle.rbl(*args)
    F1, E1, _, rho1 = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, 100, 7, 3)
    oracle.set_threads(4)
    try:
        assert oracle.get_threads() == 4
        o4 = oracle.rbl(*args)
        F4, E4, _, rho4 = oracle.rbe_forces(s.u, s.q, s.L, 0.62, 1.0, 100, 7, 3)
    finally:
        oracle.set_threads(1)
    assert np.array_equal(o1["F"], o4["F"])
    assert np.array_equal(o1["batch"], o4["batch"])
    assert np.array_equal(F1, F4) and np.array_equal(rho1, rho4) and E1 == E4
    for k in ("E_coul", "E_lj"):
        assert abs(o1[k] - o4[k]) <= 1e-12 * abs(o1[k])
    for k in ("W_coul", "W_lj", "Fsum"):
        assert np.allclose(o1[k], o4[k], rtol=0, atol=1e-11 * np.abs(o1[k]).max())
