"""Pins of the oracle's random batch list (Sec. 2.3, Eqs. 13-16, Algorithm 2).

  * Lennard-Jones special values with Lorentz-Berthelot mixing (Eqs. 2, 4):
    u(sigma_ij) = 0, minimum -eps_ij at 2^(1/6) sigma_ij with zero force;
  * the exact list (every shell member, weight 1) reproduces the explicit-image
    real-space Ewald sum of Eq. 10 (a separate code path);
  * brute force and cell list give identical lists and forces;
  * the shell estimator of Eq. 15 is unbiased, each shell member is drawn with
    probability p/N_s, and the batch is a p-subset of the shell;
  * after the correction of Eq. 16 the short-range forces sum to zero;
  * the list-size reduction matches the factor given in Sec. 2.3.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2407_09315_b300 import synth

TWO32 = 2.0 ** 32


def _pair_system(r, types=(0, 1), eps=(1.0, 4.0), sig=(1.0, 1.4), L=10.0):
    u = np.zeros((2, 3), dtype=np.uint32)
    u[0] = [100, 200, 300]
    u[1] = u[0]
    u[1, 0] = np.uint32(int(u[0, 0]) + int(round(r * TWO32 / L)))
    r_exact = (int(u[1, 0]) - int(u[0, 0])) * L / TWO32
    return u, np.zeros(2), np.array(types, np.int32), np.array(eps), np.array(sig), L, r_exact


def test_lj_special_values_with_mixing():
    eps_ij, sig_ij = 2.0, 1.2  # sqrt(1*4), (1.0+1.4)/2
    for r_target, e_ref, f_zero in ((sig_ij, 0.0, False), (2 ** (1 / 6) * sig_ij, -eps_ij, True)):
        u, q, t, eps, sig, L, r = _pair_system(r_target)
        out = oracle.rbl(u, q, t, eps, sig, L, 0.62, 1.0, 3.0, 3.5, 10, 0, 0, exact=True,
                         use_cells=False)
        # expand to first order around the exact separation
        e_lj = out["E_lj"]
        f = out["F"]
        assert out["n_core"].tolist() == [1, 1]
        slope = 24 * eps_ij * (2 * (sig_ij / r) ** 12 - (sig_ij / r) ** 6) / r  # only used as scale
        if not f_zero:
            assert abs(e_lj - e_ref) < 1e-7 * eps_ij * 48
        else:
            assert abs(e_lj - e_ref) < 1e-12
            assert np.max(np.abs(f)) < 1e-6
        assert np.allclose(f[0], -f[1], atol=1e-12)
        # repulsive inside the minimum: the force pushes atom 0 towards -x
        if not f_zero:
            assert f[0, 0] < 0


def test_exact_list_equals_real_space_ewald():
    s = synth.electrolyte(60, L=8.0, seed=4, n_types=1)
    alpha, r_cut = 0.62, 3.5
    out = oracle.rbl(s.u, s.q, s.types, np.zeros(1), np.ones(1), s.L, alpha, 1.0, 2.0, r_cut,
                     10, 0, 0, exact=True, use_cells=True)
    ref = oracle.ewald(s.u, s.q, s.L, alpha, 1.0, r_cut, 1)
    assert np.allclose(out["F"], ref["F_real"], rtol=1e-12, atol=1e-13)
    assert abs(out["E_coul"] - ref["E_real"]) < 1e-12 * abs(ref["E_real"])


def test_brute_force_and_cells_agree():
    s = synth.electrolyte(1000, L=17.1, seed=0, n_types=1)
    kw = dict(types=s.types, eps=s.eps, sig=s.sig, L=s.L, alpha=0.62, coulomb_k=1.0,
              r_core=2.0, r_cut=3.5, p=10, seed=0, step=3)
    a = oracle.rbl(s.u, s.q, use_cells=False, **kw)
    b = oracle.rbl(s.u, s.q, use_cells=True, **kw)
    for key in ("n_core", "n_shell", "n_batch", "batch"):
        assert np.array_equal(a[key], b[key]), key
    assert np.allclose(a["F"], b["F"], rtol=1e-12, atol=1e-13)
    # classification agrees with FP64 distances away from the boundaries
    x = s.x
    d = x[:, None, :] - x[None, :, :]
    d -= s.L * np.round(d / s.L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    core = (r < 2.0 - 1e-7).sum(1)
    shell = ((r > 2.0 + 1e-7) & (r < 3.5 - 1e-7)).sum(1)
    assert np.all(a["n_core"] >= core) and np.all(a["n_core"] <= (r < 2.0 + 1e-7).sum(1))
    assert np.all(a["n_shell"] >= shell)
    assert np.all(a["n_batch"] == np.minimum(a["n_shell"], 10))
    # the batch is a subset of the shell
    for i in (0, 1, 500):
        b_i = a["batch"][i][a["batch"][i] >= 0]
        assert np.all((r[i, b_i] >= 2.0 - 1e-7) & (r[i, b_i] <= 3.5 + 1e-7))
        assert len(set(b_i.tolist())) == len(b_i)


def test_shell_estimator_unbiased_and_uniform():
    s = synth.electrolyte(300, seed=6, n_types=2)
    kw = dict(types=s.types, eps=s.eps, sig=s.sig, L=s.L, alpha=0.62, coulomb_k=1.0,
              r_core=2.0, r_cut=3.5, p=6, seed=1)
    exact = oracle.rbl(s.u, s.q, exact=True, step=0, **kw)
    K = 1500
    F = np.zeros((K, s.n, 3))
    hits = np.zeros((s.n, s.n))
    for k in range(K):
        o = oracle.rbl(s.u, s.q, step=k, **kw)
        F[k] = o["F"]
        for i in range(0, s.n, 10):
            b = o["batch"][i]
            hits[i, b[b >= 0]] += 1
        assert np.array_equal(o["n_shell"], exact["n_shell"])
    z = ((F.mean(0) - exact["F"]) / (F.std(0, ddof=1) / np.sqrt(K) + 1e-300))
    big = exact["n_shell"] > 6
    zz = z[big].ravel()
    assert stats.kstest(zz, "norm").pvalue > 1e-3
    assert np.max(np.abs(zz)) < 5
    # inclusion probability p/N_s for each shell member of the sampled atoms
    for i in range(0, s.n, 10):
        Ns = exact["n_shell"][i]
        if Ns <= 6:
            continue
        members = np.nonzero(hits[i])[0]
        assert len(members) == Ns
        pr = 6.0 / Ns
        zt = (hits[i, members] - K * pr) / np.sqrt(K * pr * (1 - pr))
        assert np.max(np.abs(zt)) < 5


def test_correction_restores_zero_total_force():
    s = synth.electrolyte(400, seed=8, n_types=3)
    F, E = oracle.forces(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 50,
                         seed=2, step=4)
    assert np.linalg.norm(F.sum(0)) < 1e-10 * np.abs(F).sum()
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 2, 4)
    # the uncorrected random-batch forces do not sum to zero
    assert np.linalg.norm(o["Fsum"]) > 1e-6


def test_list_size_reduction_factor():
    s = synth.config1()
    o = oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, s.L, 0.62, 1.0, 2.0, 3.5, 10, 0, 0)
    n = s.n / s.L ** 3
    full = (o["n_core"] + o["n_shell"]).mean()
    rbl = (o["n_core"] + o["n_batch"]).mean()
    factor = 4 * np.pi * n * 3.5 ** 3 / (4 * np.pi * n * 2.0 ** 3 + 3 * 10)
    assert abs(full / rbl - factor) < 0.08 * factor


def test_selected_atoms_match_full_evaluation():
    s = synth.electrolyte(500, seed=10, n_types=2)
    kw = dict(types=s.types, eps=s.eps, sig=s.sig, L=s.L, alpha=0.62, coulomb_k=1.0,
              r_core=2.0, r_cut=3.5, p=10, seed=3, step=1)
    a = oracle.rbl(s.u, s.q, **kw)
    sel = np.array([7, 250, 499])
    b = oracle.rbl(s.u, s.q, sel=sel, want_all=False, **kw)
    assert np.array_equal(a["F"][sel], b["F"])
    assert np.array_equal(a["batch"][sel], b["batch"])
