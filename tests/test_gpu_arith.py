"""The FP64 inverse cube root of the device code (Newton-Raphson refinement
of an FP32 seed, used by the Strickler friction and the Manning form of MPM)
against CUDA's 1/cbrt: at most 2 ulp apart over 12 decades and at the
FP32-range fallback boundaries."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_inverse_cube_root_within_2_ulp():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-6, 6, 20000), rng.uniform(0.5, 2.0, 5000),
                        [1.0, 2.0, 0.1, 1e-36, 1e-40, 1e40, 3.0e38, 1.5e-38, 7.0]])
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "arith_driver")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                        os.path.join(HERE, "gpu_arith_driver.cu")], check=True)
        r = subprocess.run([exe], input="\n".join(repr(float(v)) for v in x), capture_output=True, text=True,
                           check=True)
    out = np.array([[float(t) for t in line.split()] for line in r.stdout.splitlines()])
    assert out.shape == (x.size, 3)

    def ulps(a, b):
        return np.abs(a - b) / np.spacing(np.abs(b))

    assert np.max(ulps(out[:, 1], out[:, 2])) <= 2.0
