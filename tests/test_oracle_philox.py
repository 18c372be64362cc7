"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The oracle's generator is checked against NVIDIA's cuRAND implementation of
the same published generator (curand_Philox4x32_10 from curand_philox4x32_x.h),
compiled here for the host with nvcc and run on the CPU, on random counters and
keys.  The two implementations share nothing but the publication.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

CU_SRC = r'''
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#define QUALIFIERS static inline __host__ __device__
#include <curand_philox4x32_x.h>
int main() {
    unsigned a[6];
    while (scanf("%u %u %u %u %u %u", &a[0], &a[1], &a[2], &a[3], &a[4], &a[5]) == 6) {
        uint4 c = make_uint4(a[0], a[1], a[2], a[3]);
        uint2 k = make_uint2(a[4], a[5]);
        uint4 o = curand_Philox4x32_10(c, k);
        printf("%u %u %u %u\n", o.x, o.y, o.z, o.w);
    }
    return 0;
}
'''


def _nvcc():
    for p in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return None


@pytest.mark.skipif(_nvcc() is None, reason="nvcc not available")
def test_philox_matches_curand_host_path():
    rng = np.random.default_rng(12345)
    n = 2000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64)
    # a few structured cases: zeros, all ones, small counters
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 2**32 - 1
    key[1] = 2**32 - 1
    ctr[2] = [1, 0, 0, 0]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "ph.cu")
        exe = os.path.join(d, "ph")
        open(src, "w").write(CU_SRC)
        subprocess.check_call([_nvcc(), "-O1", "-o", exe, src])
        inp = "\n".join(" ".join(str(int(v)) for v in list(c) + list(k))
                        for c, k in zip(ctr, key)) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()],
                   dtype=np.uint64)
    got = np.array([oracle.philox4x32_10(c, k) for c, k in zip(ctr, key)], dtype=np.uint64)
    assert ref.shape == got.shape
    assert np.array_equal(ref, got)


def test_philox_outputs_are_uniform_bits():
    # Counter-mode outputs over consecutive counters: every bit ~ fair coin.
    words = np.array([oracle.philox4x32_10([i, 0, 7, 1], [3, 5]) for i in range(4096)],
                     dtype=np.uint64)
    bits = ((words[:, :, None] >> np.arange(32, dtype=np.uint64)) & 1).reshape(-1, 128)
    freq = bits.mean(axis=0)
    # 4096 draws per bit: sd = 0.0078; 5 sd band
    assert np.all(np.abs(freq - 0.5) < 0.04)
