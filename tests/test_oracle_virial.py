"""Pins of the oracle's virial tensors (W = -dE/d strain at fixed fractional
coordinates; the pressure of Sec. 2.2's periodic system).

  * the trace is minus L dE/dL: central differences of the oracle's own energies
    under a uniform change of the box at fixed fixed-point coordinates, for the
    Ewald real-space and Fourier parts separately (Eq. 8) and for the erfc-Coulomb
    and LJ energies of the random batch lists with the lists unchanged;
  * the converged Coulomb sum is homogeneous of degree -1 in L, so the trace of
    the whole Ewald virial equals the total Coulomb energy, and rock salt's
    cubic symmetry makes the tensor E/3 times the identity;
  * the full tensor (not only its trace) does not depend on alpha;
  * for a cluster with exact lists inside a large box the pair virial equals
    sum_i x_i (x) F_i of the oracle's own forces (the open-boundary virial);
  * mirror and axis-permutation covariance of every component;
  * the RBE estimate averaged over many steps is unbiased for the Ewald Fourier
    virial (z-scores).
"""
import numpy as np
import pytest

import oracle

TWO32 = 2.0 ** 32


def _random_neutral(n, seed, dmin_units=None):
    rng = np.random.default_rng(seed)
    u = rng.integers(0, 2 ** 32, size=(n, 3), dtype=np.uint64).astype(np.uint32)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    q[:4] *= 2.0  # mixed valences, still neutral
    return u, q


def _ewald_energy(u, q, L, alpha, r_cut, M):
    e = oracle.ewald(u, q, L, alpha, 1.0, r_cut, M)
    return e["E_real"], e["E_recip"], e["E_self"]


def test_ewald_virial_trace_is_minus_L_dE_dL():
    n, L, alpha = 40, 6.84, 0.62
    u, q = _random_neutral(n, 3)
    r_cut = 6.2 / np.sqrt(alpha)  # converged: no pair near the cutoff matters
    M = oracle.sampler_M(L, alpha)
    Wr, Wk = oracle.ewald_virial(u, q, L, alpha, 1.0, r_cut, M)
    h = 1e-6
    Ep = _ewald_energy(u, q, L * (1 + h), alpha, r_cut, M)
    Em = _ewald_energy(u, q, L * (1 - h), alpha, r_cut, M)
    fd_real = -(Ep[0] - Em[0]) / (2 * h)
    fd_recip = -(Ep[1] - Em[1]) / (2 * h)
    assert abs(np.trace(Wr) - fd_real) < 1e-6 * abs(fd_real)
    assert abs(np.trace(Wk) - fd_recip) < 1e-6 * abs(fd_recip)
    assert np.allclose(Wr, Wr.T) and np.allclose(Wk, Wk.T)


def test_coulomb_trace_equals_energy_and_rocksalt_is_isotropic():
    n, L, alpha = 40, 6.84, 0.62
    u, q = _random_neutral(n, 4)
    r_cut = 6.2 / np.sqrt(alpha)
    M = oracle.sampler_M(L, alpha)
    Wr, Wk = oracle.ewald_virial(u, q, L, alpha, 1.0, r_cut, M)
    E = sum(_ewald_energy(u, q, L, alpha, r_cut, M))
    assert abs(np.trace(Wr + Wk) - E) < 1e-9 * abs(E)
    # rock salt, a = 1, 4^3 ions in L = 4
    g = np.arange(4)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(float)
    qs = np.where(X.sum(1) % 2 == 0, 1.0, -1.0)
    Ls = 4.0
    us = (X * (TWO32 / Ls)).astype(np.uint64).astype(np.uint32)
    Ms = oracle.sampler_M(Ls, 1.0)
    Wr, Wk = oracle.ewald_virial(us, qs, Ls, 1.0, 1.0, 6.2, Ms)
    Es = sum(_ewald_energy(us, qs, Ls, 1.0, 6.2, Ms))
    W = Wr + Wk
    assert np.allclose(W, np.eye(3) * Es / 3.0, rtol=0, atol=1e-9 * abs(Es))


def test_virial_tensor_independent_of_alpha():
    n, L = 40, 6.84
    u, q = _random_neutral(n, 5)
    Ws = []
    for alpha in (0.3, 0.62, 1.2):
        Wr, Wk = oracle.ewald_virial(u, q, L, alpha, 1.0, 6.2 / np.sqrt(alpha),
                                     oracle.sampler_M(L, alpha))
        Ws.append(Wr + Wk)
    scale = np.abs(Ws[1]).max()
    for W in Ws:
        assert np.abs(W - Ws[1]).max() < 1e-9 * scale
    # the split itself moves with alpha, so the check is not vacuous
    Wr3, _ = oracle.ewald_virial(u, q, L, 0.3, 1.0, 6.2 / np.sqrt(0.3), oracle.sampler_M(L, 0.3))
    Wr12, _ = oracle.ewald_virial(u, q, L, 1.2, 1.0, 6.2 / np.sqrt(1.2), oracle.sampler_M(L, 1.2))
    assert np.abs(Wr3 - Wr12).max() > 1e-3 * scale


def _cluster(n, seed, L, radius):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-radius, radius, 3)
        if np.linalg.norm(p) > radius or any(np.linalg.norm(p - o) < 0.8 for o in pts):
            continue
        pts.append(p)
    x = np.array(pts) + L / 2.0
    u = np.floor(x * (TWO32 / L)).astype(np.uint64).astype(np.uint32)
    return u


@pytest.mark.parametrize("part", ["coul", "lj"])
def test_cluster_pair_virial_is_sum_x_outer_f(part):
    L, n = 20.0, 12
    u = _cluster(n, 7, L, 1.6)
    x = oracle.decode(u, L)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0) if part == "coul" else np.zeros(n)
    eps = np.array([1.0, 0.7]) if part == "lj" else np.array([0.0, 0.0])
    types = (np.arange(n) % 2).astype(np.int32)
    sig = np.array([1.0, 0.9])
    # r_cut above the cluster's diameter: the exact lists hold every pair
    o = oracle.rbl(u, q, types, eps, sig, L, 0.62, 1.0, 1.2, 4.0, 3, 1, 0, exact=True)
    assert np.all(o["n_core"] + o["n_shell"] == n - 1)
    W = o["W_coul"] if part == "coul" else o["W_lj"]
    other = o["W_lj"] if part == "coul" else o["W_coul"]
    ref = x.T @ o["F"]  # sum_i x_i (x) F_i
    assert np.abs(ref).max() > 0.1
    assert np.allclose(W, ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    assert np.abs(other).max() == 0.0


def _rbl_args(n, seed):
    from paper_2407_09315_b300 import synth
    s = synth.electrolyte(n, seed=seed, charges="2:1", n_types=2)
    return s


@pytest.mark.parametrize("exact", [True, False])
def test_rbl_virial_trace_is_minus_L_dE_dL(exact):
    s = _rbl_args(700, 8)
    kw = dict(alpha=0.62, coulomb_k=1.0, r_core=2.0, r_cut=3.5, p=6, seed=4, step=2, exact=exact)

    def run(L):
        return oracle.rbl(s.u, s.q, s.types, s.eps, s.sig, L, kw["alpha"], kw["coulomb_k"],
                          kw["r_core"], kw["r_cut"], kw["p"], kw["seed"], kw["step"],
                          exact=kw["exact"])

    o = run(s.L)
    h = 2e-9
    op, om = run(s.L * (1 + h)), run(s.L * (1 - h))
    # the lists must be the same sets at L (1 +- h) (the energy is smooth only then)
    for a in (op, om):
        assert np.array_equal(a["n_core"], o["n_core"])
        assert np.array_equal(a["n_shell"], o["n_shell"])
        assert np.array_equal(a["batch"], o["batch"])
    for key, wk in (("E_coul", "W_coul"), ("E_lj", "W_lj")):
        fd = -(op[key] - om[key]) / (2 * h)
        assert abs(np.trace(o[wk]) - fd) < 1e-5 * abs(fd), (key, np.trace(o[wk]), fd)


def test_mirror_and_permutation_covariance():
    s = _rbl_args(500, 9)
    L = s.L
    u = s.u
    um = u.copy()
    um[:, 0] = ((2 ** 32 - u[:, 0].astype(np.uint64)) % 2 ** 32).astype(np.uint32)  # x -> -x
    up = np.ascontiguousarray(u[:, [1, 2, 0]])  # new axes (x, y, z) = old (y, z, x)
    args = (s.q, s.types, s.eps, s.sig)
    P = np.diag([-1.0, 1.0, 1.0])
    Pm = np.eye(3)[[1, 2, 0]]
    o, om, op = (oracle.rbl(x, *args, L, 0.62, 1.0, 2.0, 3.5, 6, 4, 2) for x in (u, um, up))
    for k in ("W_coul", "W_lj"):
        assert np.allclose(om[k], P @ o[k] @ P.T, rtol=0, atol=1e-10 * np.abs(o[k]).max())
        assert np.allclose(op[k], Pm @ o[k] @ Pm.T, rtol=0, atol=1e-10 * np.abs(o[k]).max())
    Wk, Wkm, Wkp = (oracle.rbe_virial(x, s.q, L, 0.62, 1.0, 30, 5, 1) for x in (u, um, up))
    # the mirrored box draws the same modes, so compare with the modes mirrored
    m = oracle.rbe_sample(5, 1, 30, L, 0.62)
    W = np.full(30, oracle.rbe_S(L, 0.62) / 30)
    assert np.allclose(Wk, oracle.mode_virial(u, s.q, L, 0.62, 1.0, m, W), rtol=1e-12)
    mm = m * np.array([-1, 1, 1], dtype=np.int32)
    Wmm = oracle.mode_virial(um, s.q, L, 0.62, 1.0, mm, W)
    assert np.allclose(Wmm, P @ Wk @ P.T, rtol=0, atol=1e-10 * np.abs(Wk).max())
    mp = np.ascontiguousarray(m[:, [1, 2, 0]])
    Wmp = oracle.mode_virial(up, s.q, L, 0.62, 1.0, mp, W)
    assert np.allclose(Wmp, Pm @ Wk @ Pm.T, rtol=0, atol=1e-10 * np.abs(Wk).max())


def test_rbe_virial_unbiased_for_ewald():
    n, L, alpha = 60, 6.84, 0.62
    u, q = _random_neutral(n, 10)
    M = oracle.sampler_M(L, alpha)
    _, Wk = oracle.ewald_virial(u, q, L, alpha, 1.0, 1.0, M)
    samples = np.array([oracle.rbe_virial(u, q, L, alpha, 1.0, 20, 11, st)
                        for st in range(3000)])
    mean = samples.mean(0)
    se = samples.std(0, ddof=1) / np.sqrt(len(samples))
    z = (mean - Wk) / se
    assert np.all(np.abs(z) < 4.5), z
