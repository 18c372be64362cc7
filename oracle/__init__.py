"""FP64 CPU oracle of the random-batch nonbonded step (arXiv 2407.09315).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
The arithmetic lives in ``rbmd_oracle.c`` (plain C, FP64); this module only
marshals numpy arrays through ctypes.  It shares no code with the CUDA path.

Every function cites the passage of the paper it follows; the readings taken
where the paper is silent are stated in ``rbmd_oracle.c`` beside the code.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # RBMD_ORACLE_SO points the tests at a deliberately broken build of the
        # oracle (mutation checks of the pins); unset, the source is built.
        path = os.environ.get("RBMD_ORACLE_SO") or _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32, u32, u64, dbl = C.c_int64, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_sampler_a.argtypes = [dbl, dbl]
        L.orc_sampler_a.restype = dbl
        L.orc_sampler_M.argtypes = [dbl, dbl]
        L.orc_sampler_M.restype = C.c_int
        L.orc_sampler_table.argtypes = [dbl, dbl, C.c_int, P]
        L.orc_sampler_table.restype = dbl
        L.orc_rbe_S.argtypes = [dbl, dbl]
        L.orc_rbe_S.restype = dbl
        L.orc_rbe_sample.argtypes = [u64, i64, u32, C.c_int, dbl, dbl, P]
        L.orc_full_modes.argtypes = [dbl, dbl, C.c_int, P, P]
        L.orc_full_modes.restype = i64
        L.orc_structure_factor.argtypes = [i64, P, P, dbl, i64, P, P]
        L.orc_mode_forces.argtypes = [i64, P, P, dbl, dbl, i64, P, P, i64, P, P, P, P]
        L.orc_rbe_forces.argtypes = [i64, P, P, dbl, dbl, dbl, C.c_int, u64, i64, u32,
                                     i64, P, P, P, P, P]
        L.orc_ewald.argtypes = [i64, P, P, dbl, dbl, dbl, dbl, C.c_int, P, P, P, P, P]
        L.orc_rbl_R2.argtypes = [dbl, dbl]
        L.orc_rbl_R2.restype = u64
        L.orc_rbl.argtypes = [i64, P, P, P, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32, u64,
                              i64, u32, i32, i32, i64, P, P, P, P, P, P, i32, P, P, P, P, P]
        L.orc_mode_virial.argtypes = [i64, P, P, dbl, dbl, dbl, i64, P, P, P]
        L.orc_rbe_virial.argtypes = [i64, P, P, dbl, dbl, dbl, C.c_int, u64, i64, u32, P]
        L.orc_ewald_virial.argtypes = [i64, P, P, dbl, dbl, dbl, dbl, C.c_int, P, P]
        L.orc_forces.argtypes = [i64, P, P, P, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32, i32,
                                 u64, i64, u32, i32, P, P]
        L.orc_energy_grad.argtypes = [i64, P, P, P, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32,
                                      i32, u64, i64, u32, i32, P, P, P, P, P]
        L.orc_vv.argtypes = [i64, P, P, P, P, P, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32,
                             i32, u64, i64, u32, i32, dbl, i32, dbl, dbl, i64, P]
        L.orc_langevin_normals.argtypes = [u64, u32, i64, u32, P]
        L.orc_rbe_metropolis.argtypes = [u64, i64, u32, i32, dbl, dbl, i32, P]
        L.orc_metropolis_table.argtypes = [dbl, dbl, i32, P]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n):
    """Host threads of the oracle's per-atom and per-mode loops (1 by default)."""
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _u(u):
    u = np.ascontiguousarray(u, dtype=np.uint32)
    assert u.ndim == 2 and u.shape[1] == 3
    return u


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------------------
# Philox4x32-10 (Salmon et al., SC'11)
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """ctr: 4 uint32, key: 2 uint32 -> 4 uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(o))
    return o


# --------------------------------------------------------------------------
# RBE sampling (Eq. 12, Algorithm 1 step 1)
# --------------------------------------------------------------------------
def sampler_a(L, alpha):
    return lib().orc_sampler_a(L, alpha)


def sampler_M(L, alpha):
    return lib().orc_sampler_M(L, alpha)


def sampler_table(L, alpha):
    """Returns (M, thresholds uint64[2M+1], H)."""
    M = sampler_M(L, alpha)
    T = np.zeros(2 * M + 1, dtype=np.uint64)
    H = lib().orc_sampler_table(L, alpha, M, _p(T))
    return M, T, H


def rbe_S(L, alpha):
    return lib().orc_rbe_S(L, alpha)


def rbe_sample(seed, step, P, L, alpha, replica=0):
    m = np.zeros((P, 3), dtype=np.int32)
    lib().orc_rbe_sample(seed, step, replica, P, L, alpha, _p(m))
    return m


def full_modes(L, alpha, M):
    n = lib().orc_full_modes(L, alpha, M, None, None)
    m = np.zeros((n, 3), dtype=np.int32)
    w = np.zeros(n, dtype=np.float64)
    lib().orc_full_modes(L, alpha, M, _p(m), _p(w))
    return m, w


# --------------------------------------------------------------------------
# Structure factors and mode forces (Eqs. 9, 11, 12)
# --------------------------------------------------------------------------
def structure_factor(u, q, L, m):
    u = _u(u)
    q = _d(q)
    m = np.ascontiguousarray(m, dtype=np.int32)
    rho = np.zeros((len(m), 2))
    lib().orc_structure_factor(len(u), _p(u), _p(q), L, len(m), _p(m), _p(rho))
    return rho[:, 0] + 1j * rho[:, 1]


def mode_forces(u, q, L, coulomb_k, m, W, sel=None):
    """Weighted Fourier-mode force/energy; returns (F, E, rho)."""
    u = _u(u)
    q = _d(q)
    m = np.ascontiguousarray(m, dtype=np.int32)
    W = _d(W)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
    ns = len(u) if sel is None else len(sel)
    F = np.zeros((ns, 3))
    E = C.c_double(0.0)
    rho = np.zeros((len(m), 2))
    lib().orc_mode_forces(len(u), _p(u), _p(q), L, coulomb_k, len(m), _p(m), _p(W),
                          0 if sel is None else len(sel), _p(sel), _p(F), C.byref(E), _p(rho))
    return F, E.value, rho[:, 0] + 1j * rho[:, 1]


def rbe_forces(u, q, L, alpha, coulomb_k, P, seed, step, replica=0, sel=None):
    """RBE force of one step (Eq. 12); returns (F, E_rbe, m, rho)."""
    u = _u(u)
    q = _d(q)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
    ns = len(u) if sel is None else len(sel)
    F = np.zeros((ns, 3))
    E = C.c_double(0.0)
    m = np.zeros((P, 3), dtype=np.int32)
    rho = np.zeros((P, 2))
    lib().orc_rbe_forces(len(u), _p(u), _p(q), L, alpha, coulomb_k, P, seed, step, replica,
                         0 if sel is None else len(sel), _p(sel), _p(F), C.byref(E), _p(m),
                         _p(rho))
    return F, E.value, m, rho[:, 0] + 1j * rho[:, 1]


def ewald(u, q, L, alpha, coulomb_k, r_cut, M):
    """Full Ewald (Eqs. 8, 10, 11); returns dict of forces and energies."""
    u = _u(u)
    q = _d(q)
    n = len(u)
    Fr = np.zeros((n, 3))
    Fk = np.zeros((n, 3))
    Er, Ek, Es = C.c_double(), C.c_double(), C.c_double()
    lib().orc_ewald(n, _p(u), _p(q), L, alpha, coulomb_k, r_cut, M, _p(Fr), _p(Fk),
                    C.byref(Er), C.byref(Ek), C.byref(Es))
    return dict(F_real=Fr, F_recip=Fk, E_real=Er.value, E_recip=Ek.value, E_self=Es.value)


# --------------------------------------------------------------------------
# Virial tensors (W = -dE/d strain at fixed fractional coordinates)
# --------------------------------------------------------------------------
def tensor(w6):
    """3x3 symmetric matrix of the six components xx, yy, zz, xy, xz, yz."""
    w = np.asarray(w6, dtype=np.float64)
    return np.array([[w[0], w[3], w[4]], [w[3], w[1], w[5]], [w[4], w[5], w[2]]])


def mode_virial(u, q, L, alpha, coulomb_k, m, W):
    """Virial of the weighted Fourier-mode energy (3x3)."""
    u = _u(u)
    q = _d(q)
    m = np.ascontiguousarray(m, dtype=np.int32)
    W = _d(W)
    out = np.zeros(6)
    lib().orc_mode_virial(len(u), _p(u), _p(q), L, alpha, coulomb_k, len(m), _p(m), _p(W),
                          _p(out))
    return tensor(out)


def rbe_virial(u, q, L, alpha, coulomb_k, P, seed, step, replica=0):
    """RBE estimate of the Fourier-space virial of one step (3x3)."""
    u = _u(u)
    q = _d(q)
    out = np.zeros(6)
    lib().orc_rbe_virial(len(u), _p(u), _p(q), L, alpha, coulomb_k, P, seed, step, replica,
                         _p(out))
    return tensor(out)


def ewald_virial(u, q, L, alpha, coulomb_k, r_cut, M):
    """Full Ewald virial: (real-space 3x3, Fourier 3x3)."""
    u = _u(u)
    q = _d(q)
    wr, wk = np.zeros(6), np.zeros(6)
    lib().orc_ewald_virial(len(u), _p(u), _p(q), L, alpha, coulomb_k, r_cut, M, _p(wr), _p(wk))
    return tensor(wr), tensor(wk)


# --------------------------------------------------------------------------
# Random batch list (Sec. 2.3, Eqs. 13-16, Algorithm 2)
# --------------------------------------------------------------------------
def rbl_R2(r, L):
    return lib().orc_rbl_R2(r, L)


def rbl(u, q, types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, seed, step,
        replica=0, exact=False, use_cells=True, sel=None, want_all=True):
    """Returns dict with F (uncorrected F_core + F_shell*), n_core, n_shell,
    n_batch, batch (ids ascending, -1 padded), Fsum (over all atoms, if
    want_all), E_coul, E_lj, and the virial tensors W_coul, W_lj (3x3, over all
    atoms, if want_all)."""
    u = _u(u)
    q = _d(q)
    types = np.ascontiguousarray(types, dtype=np.int32)
    eps = _d(eps)
    sig = _d(sig)
    n = len(u)
    if sel is not None:
        sel = np.ascontiguousarray(sel, dtype=np.int64)
    ns = n if sel is None else len(sel)
    F = np.zeros((ns, 3))
    nc = np.zeros(ns, dtype=np.int32)
    nsh = np.zeros(ns, dtype=np.int32)
    nb = np.zeros(ns, dtype=np.int32)
    b = np.zeros((ns, p), dtype=np.int64)
    Fs = np.zeros(3)
    Ec, El = C.c_double(), C.c_double()
    Wc, Wl = np.zeros(6), np.zeros(6)
    lib().orc_rbl(n, _p(u), _p(q), _p(types), len(eps), _p(eps), _p(sig), L, alpha, coulomb_k,
                  r_core, r_cut, p, seed, step, replica, int(exact), int(use_cells),
                  0 if sel is None else len(sel), _p(sel), _p(F), _p(nc), _p(nsh), _p(nb),
                  _p(b), int(want_all), _p(Fs), C.byref(Ec), C.byref(El), _p(Wc), _p(Wl))
    return dict(F=F, n_core=nc, n_shell=nsh, n_batch=nb, batch=b, Fsum=Fs,
                E_coul=Ec.value, E_lj=El.value, W_coul=tensor(Wc), W_lj=tensor(Wl))


def forces(u, q, types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, P, seed, step,
           replica=0, exact=False):
    """Total force of one step (RBE + RBL + Eq. 16 correction); returns (F, E[4])."""
    u = _u(u)
    q = _d(q)
    types = np.ascontiguousarray(types, dtype=np.int32)
    eps = _d(eps)
    sig = _d(sig)
    n = len(u)
    F = np.zeros((n, 3))
    E = np.zeros(4)
    lib().orc_forces(n, _p(u), _p(q), _p(types), len(eps), _p(eps), _p(sig), L, alpha,
                     coulomb_k, r_core, r_cut, p, P, seed, step, replica, int(exact), _p(F),
                     _p(E))
    return F, E


def vv(u, v, F, q, types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, P, seed, step0,
       dt, n_steps, thermostat=0, T0=1.0, tau=0.1, replica=0, exact=False, xi=0.0,
       return_xi=False):
    """Velocity-Verlet with thermostat 0 (none), 1 (Berendsen), 2 (Langevin), 3
    (Nose-Hoover, variable xi) or 4 (energy bath, xi = the bath energy E0) from
    step0; returns new (u, v, F) (and xi)."""
    u = _u(u).copy()
    v = _d(v).copy()
    F = _d(F).copy()
    q = _d(q)
    types = np.ascontiguousarray(types, dtype=np.int32)
    eps = _d(eps)
    sig = _d(sig)
    x = C.c_double(xi)
    lib().orc_vv(len(u), _p(u), _p(v), _p(F), _p(q), _p(types), len(eps), _p(eps), _p(sig),
                 L, alpha, coulomb_k, r_core, r_cut, p, P, seed, step0, replica, int(exact),
                 dt, thermostat, T0, tau, n_steps, C.byref(x))
    if return_xi:
        return u, v, F, x.value
    return u, v, F


def langevin_normals(seed, atom, step, replica=0):
    """The three standard normal deviates of the Langevin force of one atom."""
    g = np.zeros(3)
    lib().orc_langevin_normals(seed, atom, step, replica, _p(g))
    return g


def decode(u, L):
    """x = u * L / 2^32 in FP64."""
    return np.asarray(u, dtype=np.float64) * (L / 4294967296.0)


def energy_grad(u, q, types, eps, sig, L, alpha, coulomb_k, r_core, r_cut, p, P, seed, step,
                replica=0, exact=False):
    """Total potential E[4] and its gradients (dr [n,3], dq [n], deps [T], dsig [T])
    with the list weights of the step held fixed."""
    u = _u(u)
    q = _d(q)
    types = np.ascontiguousarray(types, dtype=np.int32)
    eps = _d(eps)
    sig = _d(sig)
    n = len(u)
    E = np.zeros(4)
    dr = np.zeros((n, 3))
    dq = np.zeros(n)
    de = np.zeros(len(eps))
    ds = np.zeros(len(eps))
    lib().orc_energy_grad(n, _p(u), _p(q), _p(types), len(eps), _p(eps), _p(sig), L, alpha,
                          coulomb_k, r_core, r_cut, p, P, seed, step, replica, int(exact),
                          _p(E), _p(dr), _p(dq), _p(de), _p(ds))
    return E, dr, dq, de, ds


def rbe_metropolis(seed, step, P, L, alpha, moves, replica=0):
    """Modes [P, 3] of the Metropolis chains at `step` (see orc_rbe_metropolis)."""
    m = np.zeros((P, 3), dtype=np.int32)
    lib().orc_rbe_metropolis(seed, step, replica, P, L, alpha, moves, _p(m))
    return m


def metropolis_table(L, alpha):
    """Acceptance thresholds A_k, k = 0..2M, of the Metropolis chains."""
    M = sampler_M(L, alpha)
    A = np.zeros(2 * M + 1, dtype=np.uint64)
    lib().orc_metropolis_table(L, alpha, M, _p(A))
    return A
