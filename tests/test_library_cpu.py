"""Host-side checks of the CUDA library (no GPU needed).

  * librbmd.so loads and exports every function include/rbmd.h declares;
  * the library's sampler thresholds equal the oracle's bit for bit (the two
    are written separately from the same definition, Eq. 12's factorised
    density, so every drawn mode can be compared exactly);
  * argument validation that happens before any device call.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import paper_2407_09315_b300 as rb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbmd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbmd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = rb.lib()
    names = _declared()
    assert "rbmd_init" in names and "rbmd_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert b"sm_103a" in lib.rbmd_version()


@pytest.mark.parametrize("L,alpha", [(17.1, 0.62), (79.37005259840996, 0.62),
                                     (170.99759466766966, 0.62), (368.40314986403854, 0.62),
                                     (6.0, 1.0), (2.0, 4.0)])
def test_sampler_table_matches_oracle_bitwise(L, alpha):
    M, T, H = rb.sampler_table(L, alpha)
    Mo, To, Ho = oracle.sampler_table(L, alpha)
    assert M == Mo
    assert np.array_equal(T, To)
    assert H == Ho


def test_status_strings():
    lib = rb.lib()
    for code in range(10):
        assert lib.rbmd_status_string(code)


def test_init_rejects_bad_parameters_without_device():
    lib = rb.lib()
    h = C.c_void_p()
    p = rb.Params(n_atoms=0, n_types=1, rbe_P=10, box_length=10.0, alpha=0.6, r_core=2.0,
                  r_cut=3.5, rbl_p=10)
    eps = np.ones(1)
    dummy = np.zeros(3)
    code = lib.rbmd_init(C.byref(p), rb._ptr(dummy), None, rb._ptr(dummy), None, rb._ptr(eps),
                         rb._ptr(eps), None, C.byref(h))
    assert code == 1  # RBMD_ERR_INVALID
    p.n_atoms = 10
    p.r_cut = 6.0  # >= L/2
    code = lib.rbmd_init(C.byref(p), rb._ptr(dummy), None, rb._ptr(dummy), None, rb._ptr(eps),
                         rb._ptr(eps), None, C.byref(h))
    assert code == 3  # RBMD_ERR_BOX_TOO_SMALL
    p.r_cut = 3.5
    p.rbl_p = 0
    code = lib.rbmd_init(C.byref(p), rb._ptr(dummy), None, rb._ptr(dummy), None, rb._ptr(eps),
                         rb._ptr(eps), None, C.byref(h))
    assert code == 1


def test_init_batch_rejects_mismatched_shared_parameters_without_device():
    lib = rb.lib()
    h = C.c_void_p()
    eps = np.ones(1)
    dummy = np.zeros(3)
    prm = (rb.Params * 2)()
    for r in range(2):
        prm[r] = rb.Params(n_atoms=10 + r, n_types=1, rbe_P=10, box_length=10.0 + r, alpha=0.6,
                           r_core=2.0, r_cut=3.5, rbl_p=10, seed=r, replica=r)
    prm[1].alpha = 0.7  # shared fields must agree
    code = lib.rbmd_init_batch(prm, 2, rb._ptr(dummy), None, rb._ptr(dummy), None,
                               rb._ptr(eps), rb._ptr(eps), None, C.byref(h))
    assert code == 1 and not h.value  # RBMD_ERR_INVALID, no context
    prm[1].alpha = 0.6
    prm[1].box_length = 6.0  # r_cut >= L/2 in replica 1 only
    code = lib.rbmd_init_batch(prm, 2, rb._ptr(dummy), None, rb._ptr(dummy), None,
                               rb._ptr(eps), rb._ptr(eps), None, C.byref(h))
    assert code == 3  # RBMD_ERR_BOX_TOO_SMALL
    prm[1].box_length = 11.0
    prm[0].flags = prm[1].flags = 1  # full Ewald modes: one replica only
    code = lib.rbmd_init_batch(prm, 2, rb._ptr(dummy), None, rb._ptr(dummy), None,
                               rb._ptr(eps), rb._ptr(eps), None, C.byref(h))
    assert code == 9  # RBMD_ERR_UNSUPPORTED
    code = lib.rbmd_init_batch(prm, 0, rb._ptr(dummy), None, rb._ptr(dummy), None,
                               rb._ptr(eps), rb._ptr(eps), None, C.byref(h))
    assert code == 1


@pytest.mark.parametrize("L,alpha", [(17.1, 0.62), (170.99759466766966, 0.62), (8.0, 0.62),
                                     (368.40314986403854, 0.62)])
def test_metropolis_table_matches_oracle_bitwise(L, alpha):
    A = rb.metropolis_table(L, alpha)
    Ao = oracle.metropolis_table(L, alpha)
    assert A.dtype == np.uint64 and np.array_equal(A, Ao)
