"""The bounds-checked build (librbmd_checked.so, -DRBMD_CHECKED: every list and
cell index of the RBL kernels checked on the device, an index out of range
latched as RBMD_ERR_BOUNDS instead of being used) gives the default build's
results on the calls of tests/checked_worker.py: no error latched, integer lists
identical, forces, trajectories, energies and gradients within rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(lib, out):
    env = dict(os.environ)
    if lib:
        env["RBMD_LIBRARY"] = lib
    subprocess.run([sys.executable, os.path.join(HERE, "checked_worker.py"), out], env=env,
                   check=True, timeout=600)
    return dict(np.load(out))


def test_checked_build_matches_default(tmp_path):
    from paper_2407_09315_b300 import build

    checked = build.build(checked=True)
    a = _run(None, str(tmp_path / "default.npz"))
    b = _run(checked, str(tmp_path / "checked.npz"))
    assert a.keys() == b.keys()
    for k in a:
        if k.endswith("_lists"):
            assert np.array_equal(a[k], b[k]), k
        else:
            scale = max(np.abs(a[k]).max(), 1e-30)
            assert np.abs(a[k] - b[k]).max() <= 1e-5 * scale, k
