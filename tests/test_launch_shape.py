"""The FP32 solve pass's launch shape as bench.py counts it (strips of 30
columns, runs of rows: the solves and projections per cell in its roofline
depend on them) equals the library's own choice (march_shape in
csrc/sve_march.cuh), on the benchmark grids, the ensemble's range, narrow
grids and several SM counts.  The C++ side is compiled for the host and run
on the CPU: no GPU."""
from __future__ import annotations

import importlib.util
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

GRIDS = [(1024, 512), (8192, 4096), (4096, 2048), (4000, 4000), (1000, 1000), (2048, 1024), (128, 64),
         (1024, 512), (97, 45), (31, 7), (33, 9), (30, 1), (61, 300), (7, 5000)]
NSMS = [152, 148, 132, 1]


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _library_shapes(cases):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    csrc = os.path.join(ROOT, "paper_1307_0491_gb300", "csrc")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "launch_shape")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I", csrc, "-I",
                        os.path.join(ROOT, "include"), "-o", exe, os.path.join(HERE, "launch_shape_driver.cu")],
                       check=True)
        r = subprocess.run([exe], input="\n".join(f"{nx} {ny} {nsm}" for nx, ny, nsm in cases),
                           capture_output=True, text=True, check=True)
    return [tuple(int(t) for t in line.split()) for line in r.stdout.splitlines()]


def test_bench_counts_the_library_launch_shape():
    bench = _bench()
    cases = [(nx, ny, nsm) for nx, ny in GRIDS for nsm in NSMS]
    got = _library_shapes(cases)
    assert len(got) == len(cases)
    for (nx, ny, nsm), (strips, rows, chunks, tasks, blocks) in zip(cases, got):
        assert bench.march_shape(nx, ny, nsm) == (strips, chunks), (nx, ny, nsm)
        # every row of every strip is covered once
        assert 4 <= rows <= 32 and chunks * rows >= ny > (chunks - 1) * rows, (nx, ny, nsm, rows, chunks)
        assert tasks == strips * chunks and blocks == -(-tasks // 4)
