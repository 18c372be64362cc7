"""B300 random-batch molecular dynamics (arXiv 2407.09315): Python binding.

The compute path is the CUDA library ``librbmd.so`` (C ABI, ``include/rbmd.h``);
this module only marshals arguments through ctypes.  PyTorch supplies device
memory and the current CUDA stream.  There is no CPU fallback: if the library
is missing the import of :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# RBMD_LIBRARY selects another build of the library (the bounds-checked
# librbmd_checked.so, for debugging); by default the in-tree librbmd.so
LIB_PATH = os.environ.get("RBMD_LIBRARY") or os.path.join(_HERE, "librbmd.so")

FP32, FP64 = 0, 1
FULL_EWALD_MODES, RBL_EXACT, NO_RBE, NO_RBL, PAIR_TABLE, METROPOLIS_MODES = 1, 2, 4, 8, 16, 32

STATUS = {
    0: "RBMD_OK", 1: "RBMD_ERR_INVALID", 2: "RBMD_ERR_NOT_NEUTRAL",
    3: "RBMD_ERR_BOX_TOO_SMALL", 4: "RBMD_ERR_OOM", 5: "RBMD_ERR_CUDA",
    6: "RBMD_ERR_CELL_OVERFLOW", 7: "RBMD_ERR_NONFINITE", 8: "RBMD_ERR_TIMEOUT",
    9: "RBMD_ERR_UNSUPPORTED", 10: "RBMD_ERR_BOUNDS",
}


class RBMDError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__("%s (%d)%s" % (STATUS.get(code, "?"), code, (": " + what) if what else ""))


class Params(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int64), ("n_types", C.c_int32), ("rbe_P", C.c_int32),
        ("box_length", C.c_double), ("alpha", C.c_double), ("r_core", C.c_double),
        ("r_cut", C.c_double), ("rbl_p", C.c_int32), ("thermostat", C.c_int32),
        ("coulomb_k", C.c_double), ("dt", C.c_double), ("temperature", C.c_double),
        ("tau_T", C.c_double), ("seed", C.c_uint64), ("replica", C.c_uint32),
        ("precision", C.c_int32), ("flags", C.c_uint32), ("cell_div", C.c_int32),
        ("mh_moves", C.c_int32), ("skin", C.c_double),
    ]


class EnergyTerms(C.Structure):
    _fields_ = [
        ("e_coul_real", C.c_double), ("e_lj", C.c_double), ("e_rbe", C.c_double),
        ("e_self", C.c_double), ("e_potential", C.c_double), ("e_kinetic", C.c_double),
        ("temperature", C.c_double), ("S", C.c_double), ("fsum_short", C.c_double * 3),
        ("step", C.c_int64), ("max_shell", C.c_int32), ("max_cell", C.c_int32),
        ("virial", C.c_double * 6), ("virial_coul_real", C.c_double), ("virial_lj", C.c_double),
        ("virial_rbe", C.c_double), ("pressure", C.c_double),
    ]


_lib = None


def lib():
    """Load librbmd.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("librbmd.so is missing: run `python -m paper_2407_09315_b300.build` "
                           "(or __graft_entry__.build()) first")
    L = C.CDLL(LIB_PATH)
    P, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "rbmd_status_string": ([C.c_int], C.c_char_p),
        "rbmd_version": ([], C.c_char_p),
        "rbmd_init": ([C.POINTER(Params), P, P, P, P, P, P, P, C.POINTER(P)], C.c_int),
        "rbmd_init_batch": ([C.POINTER(Params), i32, P, P, P, P, P, P, P, C.POINTER(P)], C.c_int),
        "rbmd_replica_count": ([P], i32),
        "rbmd_candidate_rebuilds": ([P], i64),
        "rbmd_init_slab": ([C.POINTER(Params), i64, i64, P, P, P, P, P, P, P, P, C.POINTER(P)],
                           C.c_int),
        "rbmd_rbe_rho_partial": ([P, i64, P], C.c_int),
        "rbmd_rho_acc_add": ([P, P, i64], None),
        "rbmd_rbe_forces_rho": ([P, i64, P, P, C.c_int], C.c_int),
        "rbmd_rbl_forces_slab": ([P, i64, P, C.c_int, P], C.c_int),
        "rbmd_add_correction": ([P, P, P], C.c_int),
        "rbmd_set_tiles": ([P, i32, i32, i32], C.c_int),
        "rbmd_get_tiles": ([P, P], C.c_int),
        "rbmd_autotune": ([P, i64, P], C.c_int),
        "rbmd_set_pair_table": ([P, i32], C.c_int),
        "rbmd_get_thermostat": ([P, P], C.c_int),
        "rbmd_set_thermostat": ([P, P], C.c_int),
        "rbmd_pair_table": ([dbl, dbl, i32, C.POINTER(i32), C.POINTER(dbl), P], C.c_int),
        "rbmd_metropolis_table": ([dbl, dbl, P], C.c_int),
        "rbmd_energy_batch": ([P, i64, C.POINTER(EnergyTerms)], C.c_int),
        "rbmd_destroy": ([P], None),
        "rbmd_rbe_forces": ([P, i64, P, C.c_int], C.c_int),
        "rbmd_rbl_forces": ([P, i64, P, C.c_int], C.c_int),
        "rbmd_forces": ([P, i64, P, C.c_int], C.c_int),
        "rbmd_forces_host": ([P, P, P, i64], C.c_int),
        "rbmd_step": ([P, i64], C.c_int),
        "rbmd_energy": ([P, i64, C.POINTER(EnergyTerms)], C.c_int),
        "rbmd_energy_backward": ([P, i64, dbl, P, P, P, P], C.c_int),
        "rbmd_get_state": ([P, P, P, C.POINTER(i64)], C.c_int),
        "rbmd_set_state": ([P, P, P, i64], C.c_int),
        "rbmd_get_state_u": ([P, P, P, C.POINTER(i64)], C.c_int),
        "rbmd_set_state_u": ([P, P, P, i64], C.c_int),
        "rbmd_sync": ([P], C.c_int),
        "rbmd_rbe_mode_count": ([P], i64),
        "rbmd_rbe_modes": ([P, i64, P, P], C.c_int),
        "rbmd_rbl_lists": ([P, i64, P, P, P], C.c_int),
        "rbmd_sampler_table": ([dbl, dbl, C.POINTER(i32), P, C.POINTER(dbl)], C.c_int),
        "rbmd_debug_latch_error": ([P, i32], C.c_int),
        "rbmd_profile": ([P, C.c_int], C.c_int),
        "rbmd_profile_read": ([P, P, C.POINTER(i64), C.c_int], C.c_int),
        "rbmd_step_kernel_count": ([P], i32),
        "rbmd_rebuild_kernel_count": ([P], i32),
        "rbmd_profile_read_grad": ([P, P, P, P, C.c_int], C.c_int),
        "rbmd_set_charges": ([P, P], C.c_int),
        "rbmd_set_lj": ([P, P, P], C.c_int),
        "rbmd_rbe_forces_noalloc": ([P, P, i64, dbl, dbl, dbl, i32, C.c_uint64, i64, C.c_uint32,
                                     P, P], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(code: int, what: str = ""):
    if code != 0:
        raise RBMDError(code, what)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def sampler_table(box_length: float, alpha: float):
    """Inverse-CDF thresholds of the mode sampler: (M, uint64[2M+1], H)."""
    M = C.c_int32(0)
    _check(lib().rbmd_sampler_table(box_length, alpha, C.byref(M), None, None))
    T = np.zeros(2 * M.value + 1, dtype=np.uint64)
    H = C.c_double(0.0)
    _check(lib().rbmd_sampler_table(box_length, alpha, C.byref(M), _ptr(T), C.byref(H)))
    return M.value, T, H.value


def metropolis_table(box_length, alpha):
    """Acceptance thresholds A_k (uint64 [2M + 1]) of the Metropolis mode chains."""
    M, _, _ = sampler_table(box_length, alpha)
    A = np.zeros(2 * M + 1, dtype=np.uint64)
    _check(lib().rbmd_metropolis_table(box_length, alpha, _ptr(A)), "metropolis_table")
    return A


def pair_table(alpha, r_cut, n):
    """The erfc-Coulomb look-up table: (i0, inv_h, coef [n, 2, 4]) (see rbmd.h)."""
    i0 = C.c_int32(0)
    inv_h = C.c_double(0.0)
    coef = np.zeros((n, 2, 4), dtype=np.float64)
    _check(lib().rbmd_pair_table(alpha, r_cut, n, C.byref(i0), C.byref(inv_h), _ptr(coef)),
           "pair_table")
    return i0.value, inv_h.value, coef


def rho_acc_add(total, part):
    """total += part for exact structure-factor sums (int64 numpy [P, 4], the
    128-bit words of rbmd_rbe_rho_partial); in place, returns total."""
    t = np.ascontiguousarray(total, dtype=np.int64)
    q = np.ascontiguousarray(part, dtype=np.int64)
    if t.shape != q.shape or t.ndim != 2 or t.shape[1] != 4:
        raise ValueError("acc arrays must be int64 [P, 4] of one shape")
    lib().rbmd_rho_acc_add(_ptr(t), _ptr(q), t.shape[0])
    if t is not total:
        total[...] = t
    return total


def rbe_forces_noalloc(u, charge, box_length, *, alpha, coulomb_k, P, seed, step, out,
                       replica=0, stream=None):
    """RBE force without a context or any device allocation (FP32).

    u: CUDA int32/uint32 tensor [N, 3] of fixed-point positions; charge: CUDA
    float32 [N]; out: CUDA float32 [N, 3], overwritten.  All three must be
    contiguous and on one device.  For callers that cannot allocate device
    memory; all scratch is a fixed static device array.
    """
    import torch

    ok_u = getattr(torch, "uint32", None)
    if not all(isinstance(t, torch.Tensor) and t.is_cuda for t in (u, charge, out)):
        raise ValueError("u, charge and out must be CUDA tensors")
    if not (u.device == charge.device == out.device):
        raise ValueError("u, charge and out must be on one device")
    if not all(t.is_contiguous() for t in (u, charge, out)):
        raise ValueError("u, charge and out must be contiguous")
    if u.dim() != 2 or u.shape[1] != 3 or u.dtype not in (torch.int32, ok_u):
        raise ValueError("u must be an int32 or uint32 tensor of shape [N, 3]")
    n = int(u.shape[0])
    if charge.dtype != torch.float32 or tuple(charge.shape) != (n,):
        raise ValueError("charge must be a float32 tensor of shape [N]")
    if out.dtype != torch.float32 or tuple(out.shape) != (n, 3):
        raise ValueError("out must be a float32 tensor of shape [N, 3]")
    with torch.cuda.device(out.device):
        if stream is None:
            stream = torch.cuda.current_stream(out.device)
        _check(lib().rbmd_rbe_forces_noalloc(_ptr(u), _ptr(charge), n, box_length, alpha,
                                             coulomb_k, P, seed, step, replica, _ptr(out),
                                             C.c_void_p(stream.cuda_stream)),
               "rbe_forces_noalloc")
    return out


class RBMD:
    """One simulation context on the current CUDA device and stream.

    pos, vel: CUDA tensors [N, 3] (float32 for FP32 contexts, float64 for FP64);
    charge: CUDA tensor [N] of the same dtype; types: CUDA int32 tensor [N] or None;
    eps, sigma: per-type LJ parameters (host sequences).

    A batch of R independent replicas is made by giving box_length as a sequence
    of R boxes and n_atoms as the R atom counts (seed, replica and temperature may
    be scalars or length-R sequences); pos, charge, vel and types are then the
    replicas' arrays concatenated in order.
    """

    def __init__(self, pos, charge, eps, sigma, *, box_length, alpha=0.62, r_core=2.0,
                 r_cut=3.5, rbl_p=10, rbe_P=100, coulomb_k=1.0, dt=0.001, temperature=1.0,
                 tau_T=0.1, thermostat=0, seed=0, replica=0, precision=FP32, flags=0,
                 cell_div=0, vel=None, types=None, stream=None, n_atoms=None, mh_moves=0,
                 skin=0.0, slab=None):
        import torch

        self._torch = torch
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.device = pos.device
        n = pos.shape[0]
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        self.n = n
        self.n_types = len(eps)
        self.p = rbl_p
        batched = np.ndim(box_length) > 0
        boxes = list(box_length) if batched else [box_length]
        R = len(boxes)
        sizes = list(n_atoms) if batched else [n]
        if len(sizes) != R or sum(sizes) != n:
            raise ValueError("n_atoms must list one size per box and sum to pos.shape[0]")

        def per(v):
            return list(v) if np.ndim(v) > 0 else [v] * R

        seeds, reps, temps = per(seed), per(replica), per(temperature)
        self.R = R
        self.sizes = sizes
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.box_lengths = boxes
        prm = (Params * R)()
        for r in range(R):
            prm[r] = Params(n_atoms=sizes[r], n_types=len(eps), rbe_P=rbe_P,
                            box_length=boxes[r], alpha=alpha, r_core=r_core, r_cut=r_cut,
                            rbl_p=rbl_p, thermostat=thermostat, coulomb_k=coulomb_k, dt=dt,
                            temperature=temps[r], tau_T=tau_T, seed=seeds[r],
                            replica=reps[r], precision=precision, flags=flags,
                            cell_div=cell_div, mh_moves=mh_moves, skin=skin)
        self.params = prm[0]
        self._params = prm
        pos = pos.to(self.dtype).contiguous()
        charge = charge.to(self.dtype).contiguous()
        vel = None if vel is None else vel.to(self.dtype).contiguous()
        types = None if types is None else types.to(torch.int32).contiguous()
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = C.c_void_p()
        self.slab = slab
        if slab is not None:
            # (n_owned, n_global, gid): a slab context of a spatial decomposition
            n_owned, n_global, gid = slab
            gid = gid.to(self.device, torch.int32).contiguous()
            self.n_owned = int(n_owned)
            _check(lib().rbmd_init_slab(prm, int(n_owned), int(n_global), _ptr(gid), _ptr(pos),
                                        _ptr(vel), _ptr(charge), _ptr(types), _ptr(eps),
                                        _ptr(sigma), C.c_void_p(stream.cuda_stream), C.byref(h)),
                   "rbmd_init_slab")
            self._gid = gid
        else:
            self.n_owned = n
            _check(lib().rbmd_init_batch(prm, R, _ptr(pos), _ptr(vel), _ptr(charge), _ptr(types),
                                         _ptr(eps), _ptr(sigma), C.c_void_p(stream.cuda_stream),
                                         C.byref(h)), "rbmd_init_batch")
        self._h = h
        # the context copied the inputs on `stream`; once that work is done the
        # caller's tensors (and any converted copies made here) can go
        stream.synchronize()

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().rbmd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _new3(self):
        return self._torch.empty((self.n, 3), dtype=self.dtype, device=self.device)

    # -- forces -----------------------------------------------------------
    def rbe_forces(self, step, out=None, accumulate=False):
        out = self._new3() if out is None else out
        _check(lib().rbmd_rbe_forces(self._h, step, _ptr(out), int(accumulate)), "rbe_forces")
        return out

    def rbl_forces(self, step, out=None, accumulate=False):
        out = self._new3() if out is None else out
        _check(lib().rbmd_rbl_forces(self._h, step, _ptr(out), int(accumulate)), "rbl_forces")
        return out

    def forces(self, step, out=None, accumulate=False):
        out = self._new3() if out is None else out
        _check(lib().rbmd_forces(self._h, step, _ptr(out), int(accumulate)), "forces")
        return out

    # -- spatial decomposition (slab contexts) -----------------------------
    def rho_partial(self, step):
        """Exact structure-factor sums of the owned atoms (int64 numpy [R*P, 4])."""
        acc = np.zeros((self.R * self.mode_count(), 4), dtype=np.int64)
        _check(lib().rbmd_rbe_rho_partial(self._h, step, _ptr(acc)), "rbe_rho_partial")
        return acc

    def forces_rho(self, step, acc, out=None, accumulate=False):
        """RBE force of the owned atoms from summed structure factors (rho_partial
        summed over ranks with rho_acc_add)."""
        out = self._new3() if out is None else out
        acc = np.ascontiguousarray(acc, dtype=np.int64)
        _check(lib().rbmd_rbe_forces_rho(self._h, step, _ptr(acc), _ptr(out), int(accumulate)),
               "rbe_forces_rho")
        return out

    def rbl_forces_slab(self, step, out=None, accumulate=False):
        """RBL force of the owned atoms without the momentum correction, and the sum
        of those forces (numpy [3])."""
        out = self._new3() if out is None else out
        fsum = np.zeros(3)
        _check(lib().rbmd_rbl_forces_slab(self._h, step, _ptr(out), int(accumulate), _ptr(fsum)),
               "rbl_forces_slab")
        return out, fsum

    def add_correction(self, force, fsum_total):
        """force (owned rows) += -fsum_total / n_global (Eq. 16 over all ranks)."""
        f = np.ascontiguousarray(fsum_total, dtype=np.float64)
        _check(lib().rbmd_add_correction(self._h, _ptr(force), _ptr(f)), "add_correction")
        return force

    def forces_host(self, pos, out=None, step=0):
        """Host positions in (they become the state, as set_state), host forces out:
        rbmd_forces_host.  pos: CPU tensor [N, 3] of the context's dtype (pinned
        memory lets the copies overlap the kernels); out: CPU tensor or None."""
        t = self._torch
        if pos.device.type != "cpu" or pos.dtype != self.dtype or not pos.is_contiguous():
            raise ValueError("pos must be a contiguous CPU tensor of the context's dtype")
        if out is None:
            out = t.empty((self.n, 3), dtype=self.dtype, pin_memory=pos.is_pinned())
        _check(lib().rbmd_forces_host(self._h, _ptr(pos), _ptr(out), step), "forces_host")
        return out

    # -- dynamics ---------------------------------------------------------
    def step(self, n_steps=1):
        _check(lib().rbmd_step(self._h, n_steps), "step")

    @staticmethod
    def _terms(e) -> dict:
        d = {k: getattr(e, k) for k, _ in EnergyTerms._fields_}
        d["fsum_short"] = list(e.fsum_short)
        w = list(e.virial)
        d["virial"] = np.array([[w[0], w[3], w[4]], [w[3], w[1], w[5]], [w[4], w[5], w[2]]])
        return d

    def energy(self, step) -> dict:
        e = EnergyTerms()
        _check(lib().rbmd_energy(self._h, step, C.byref(e)), "energy")
        return self._terms(e)

    def energy_batch(self, step) -> list:
        """Energies of every replica (list of dicts, replica order)."""
        e = (EnergyTerms * self.R)()
        _check(lib().rbmd_energy_batch(self._h, step, e), "energy_batch")
        return [self._terms(x) for x in e]

    def energy_backward(self, step, grad_out=1.0, want_pos=True, want_q=True, want_lj=True):
        t = self._torch
        dpos = t.empty((self.n, 3), dtype=self.dtype, device=self.device) if want_pos else None
        dq = t.empty((self.n,), dtype=self.dtype, device=self.device) if want_q else None
        de = np.zeros(self.n_types) if want_lj else None
        ds = np.zeros(self.n_types) if want_lj else None
        _check(lib().rbmd_energy_backward(self._h, step, grad_out, _ptr(dpos), _ptr(dq),
                                          _ptr(de), _ptr(ds)), "energy_backward")
        return dpos, dq, de, ds

    def set_charges(self, q):
        q = q.to(self.device, self.dtype).contiguous()
        _check(lib().rbmd_set_charges(self._h, _ptr(q)), "set_charges")

    def set_lj(self, eps, sigma):
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        _check(lib().rbmd_set_lj(self._h, _ptr(eps), _ptr(sigma)), "set_lj")

    # -- state ------------------------------------------------------------
    def get_state(self):
        pos, vel = self._new3(), self._new3()
        st = C.c_int64(0)
        _check(lib().rbmd_get_state(self._h, _ptr(pos), _ptr(vel), C.byref(st)), "get_state")
        return pos, vel, st.value

    def set_state(self, pos=None, vel=None, step=0):
        _check(lib().rbmd_set_state(self._h, _ptr(pos), _ptr(vel), step), "set_state")

    def get_state_u(self):
        u = self._torch.empty((self.n, 3), dtype=self._torch.int32, device=self.device)
        vel = self._new3()
        st = C.c_int64(0)
        _check(lib().rbmd_get_state_u(self._h, _ptr(u), _ptr(vel), C.byref(st)), "get_state_u")
        return u, vel, st.value

    def set_state_u(self, u, vel=None, step=0):
        """u: uint32 fixed-point coordinates [N, 3] (numpy or an int32 tensor view)."""
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.uint32)
            ut = self._torch.from_numpy(u.view(np.int32)).to(self.device)
        else:
            ut = u.contiguous()
        if vel is not None and isinstance(vel, np.ndarray):
            vel = self._torch.from_numpy(np.ascontiguousarray(vel)).to(self.device, self.dtype)
        _check(lib().rbmd_set_state_u(self._h, _ptr(ut), _ptr(vel), step), "set_state_u")
        self._torch.cuda.current_stream(self.device).synchronize()

    def thermostat_state(self):
        """Nose-Hoover variable xi, or the energy bath's E0 (NaN until the first
        step takes it), of every replica (numpy [R])."""
        xi = np.zeros(self.R)
        _check(lib().rbmd_get_thermostat(self._h, _ptr(xi)), "get_thermostat")
        return xi

    def set_thermostat_state(self, xi):
        xi = np.ascontiguousarray(np.atleast_1d(xi), dtype=np.float64)
        _check(lib().rbmd_set_thermostat(self._h, _ptr(xi)), "set_thermostat")

    def sync(self):
        _check(lib().rbmd_sync(self._h), "sync")

    def candidate_rebuilds(self) -> int:
        """Rebuilds of the step's neighbour candidate lists so far (0: lists off)."""
        return int(lib().rbmd_candidate_rebuilds(self._h))

    # -- inspection -------------------------------------------------------
    def mode_count(self) -> int:
        return lib().rbmd_rbe_mode_count(self._h)

    def rbe_modes(self, step):
        """Modes [R*P, 3] and structure factors [R*P] (replica blocks of P)."""
        P = self.mode_count() * self.R
        m = np.zeros((P, 3), dtype=np.int32)
        rho = np.zeros((P, 2), dtype=np.float64)
        _check(lib().rbmd_rbe_modes(self._h, step, _ptr(m), _ptr(rho)), "rbe_modes")
        return m, rho[:, 0] + 1j * rho[:, 1]

    def rbl_lists(self, step):
        t = self._torch
        nc = t.empty((self.n,), dtype=t.int32, device=self.device)
        ns = t.empty((self.n,), dtype=t.int32, device=self.device)
        b = t.empty((self.n, self.p), dtype=t.int32, device=self.device)
        _check(lib().rbmd_rbl_lists(self._h, step, _ptr(nc), _ptr(ns), _ptr(b)), "rbl_lists")
        return nc, ns, b

    # -- measurement ------------------------------------------------------
    PROFILE_STAGES = ("kick_drift", "cell_sort", "rbl_scan", "rbl_select", "rbl_force",
                      "f_corr", "rbe_sample", "rho_partial", "rho_final", "rbe_force",
                      "kick_thermo")

    def profile(self, enable=True):
        _check(lib().rbmd_profile(self._h, int(enable)), "profile")

    def profile_read(self, reset=False):
        ms = np.zeros(len(self.PROFILE_STAGES))
        n = C.c_int64(0)
        _check(lib().rbmd_profile_read(self._h, _ptr(ms), C.byref(n), int(reset)), "profile_read")
        return dict(zip(self.PROFILE_STAGES, ms.tolist())), n.value

    FWD_STAGES = ("rbe", "cell_sort", "rbl_pairs", "sums")
    BWD_STAGES = ("lists", "rbe_rho", "init", "rbl_adjoint", "rbe_adjoint")

    def profile_read_grad(self, reset=False):
        """Accumulated stage times (ms) of rbmd_energy and rbmd_energy_backward while
        profiling: (forward dict, backward dict, (forward calls, backward calls))."""
        f = np.zeros(len(self.FWD_STAGES))
        b = np.zeros(len(self.BWD_STAGES))
        n = np.zeros(2, dtype=np.int64)
        _check(lib().rbmd_profile_read_grad(self._h, _ptr(f), _ptr(b), _ptr(n), int(reset)),
               "profile_read_grad")
        return (dict(zip(self.FWD_STAGES, f.tolist())), dict(zip(self.BWD_STAGES, b.tolist())),
                (int(n[0]), int(n[1])))

    def set_tiles(self, cell_div, rho_tile, rho_mode_tile):
        _check(lib().rbmd_set_tiles(self._h, cell_div, rho_tile, rho_mode_tile), "set_tiles")

    def tiles(self):
        """(cell_div, rho_tile, rho_mode_tile, pair_table) in use."""
        out = np.zeros(4, dtype=np.int32)
        _check(lib().rbmd_get_tiles(self._h, _ptr(out)), "get_tiles")
        return tuple(int(x) for x in out)

    def set_pair_table(self, on=True):
        _check(lib().rbmd_set_pair_table(self._h, int(bool(on))), "set_pair_table")

    def autotune(self, step=0):
        """Time the tile-shape and pair-table candidates on the current state and keep
        the fastest; returns tiles()."""
        out = np.zeros(4, dtype=np.int32)
        _check(lib().rbmd_autotune(self._h, step, _ptr(out)), "autotune")
        return tuple(int(x) for x in out)

    def step_kernel_count(self) -> int:
        return lib().rbmd_step_kernel_count(self._h)

    def rebuild_kernel_count(self) -> int:
        """Kernels a step adds when it rebuilds the candidate lists."""
        return lib().rbmd_rebuild_kernel_count(self._h)

    def debug_latch_error(self, code):
        _check(lib().rbmd_debug_latch_error(self._h, code))
