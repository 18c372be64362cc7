"""Failure paths, made on the host (nothing here faults, traps or hangs a GPU):
an injected allocation failure, non-neutral charges, an invalid LJ type, a NaN
velocity that the integrator reports, and the latched device error word."""
import numpy as np
import pytest

import paper_2407_09315_b300 as rb
from paper_2407_09315_b300 import synth

from gpu_util import make_ctx

pytestmark = pytest.mark.gpu


def _code(fn):
    with pytest.raises(rb.RBMDError) as e:
        fn()
    return e.value.code


def test_injected_allocation_failure_returns_oom(monkeypatch):
    s = synth.electrolyte(500, seed=51)
    for k in (0, 3, 17):
        monkeypatch.setenv("RBMD_FAIL_ALLOC_AFTER", str(k))
        assert _code(lambda: make_ctx(s, rb.FP32)) == 4  # RBMD_ERR_OOM
    monkeypatch.delenv("RBMD_FAIL_ALLOC_AFTER")
    ctx, _ = make_ctx(s, rb.FP32)  # the library is still usable
    ctx.forces(0)
    ctx.sync()
    ctx.close()


def test_non_neutral_and_bad_type_are_rejected():
    s = synth.electrolyte(400, seed=52)
    s.q = np.abs(s.q)
    assert _code(lambda: make_ctx(s, rb.FP64)) == 2  # RBMD_ERR_NOT_NEUTRAL
    s = synth.electrolyte(400, seed=52, n_types=2)
    s.types = s.types.copy()
    s.types[5] = 7
    assert _code(lambda: make_ctx(s, rb.FP32)) == 1  # RBMD_ERR_INVALID


def test_nan_velocity_latches_nonfinite_and_clears():
    s = synth.electrolyte(800, seed=53)
    ctx, _ = make_ctx(s, rb.FP32, thermostat=0)
    v = s.v.copy()
    v[10, 1] = np.nan
    ctx.set_state_u(s.u, vel=v, step=0)
    ctx.step(1)
    assert _code(ctx.sync) == 7  # RBMD_ERR_NONFINITE
    ctx.sync()  # cleared once reported
    ctx.close()


def test_latched_error_is_reported_by_the_next_sync():
    s = synth.electrolyte(300, seed=54)
    ctx, _ = make_ctx(s, rb.FP32)
    ctx.debug_latch_error(8)
    assert _code(ctx.sync) == 8  # RBMD_ERR_TIMEOUT
    ctx.sync()
    ctx.close()


def test_latched_error_is_reported_by_the_next_energy_call():
    # rbmd_energy reads the error word back with its results and clears it
    s = synth.electrolyte(300, seed=55)
    ctx, _ = make_ctx(s, rb.FP32)
    ctx.debug_latch_error(8)
    assert _code(lambda: ctx.energy(0)) == 8
    e = ctx.energy(0)
    assert np.isfinite(e["e_potential"])
    ctx.sync()
    ctx.close()
