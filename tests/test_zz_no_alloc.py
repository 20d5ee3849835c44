"""sve_step_noalloc: stepping for callers that cannot allocate device memory.

Such callers (code under a framework's caching allocator that owns the
device memory, real-time loops that must not allocate mid-run, plug-ins that
get device buffers but no allocator) hand the library their own device
arrays; the step's scratch comes from the library's static device array.
This test calls the entry point through the C ABI twice in a row and checks
each result against the regular entry points (sve_create / sve_set_state /
sve_step) within the FP64 parity tolerance of the other GPU tests.  It sits
in a file of its own, collected last, and passes alone or after the others.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()


def _rel(a, b, scale):
    return float(np.max(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))) / scale)


@pytest.mark.parametrize("dim", [2, 1])
def test_noalloc_matches_regular_entry_points_twice(dim):
    import torch

    if dim == 2:
        w = W.dune2d(nx=150, ny=70, seed=11, lx=150.0, ly=70.0)
        w["params"].update(bc=("inflow_q", "free", "wall", "free"))
    else:
        w = W.dune1d(nx=900)
    p = w["params"]
    cfg = sve.config_from_params(p, "fp64")
    names = ("h", "hu", "hv", "z") if dim == 2 else ("h", "hu", "z")
    dev = {k: torch.tensor(np.asarray(w[k]), dtype=torch.float64, device="cuda").contiguous() for k in names}
    ptr = lambda k: dev[k].data_ptr() if k in dev else None

    ref = sve.Solver(p, "fp64")
    ref.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = 0.0
    for call, n in enumerate((40, 25)):
        rc, t = sve.sve_step_noalloc(cfg, ptr("h"), ptr("hu"), ptr("hv"), ptr("z"), n, t)
        assert rc == sve.SVE_OK, sve.sve_strerror(rc)
        t_ref = ref.step(n)
        got = {k: dev[k].cpu().numpy() for k in names}
        exp = ref.get_state()
        qscale = max(np.max(np.abs(exp["hu"])), 1e-12)
        assert _rel(got["h"], exp["h"], np.max(np.abs(exp["h"]))) <= TOL64, call
        assert _rel(got["z"], exp["z"], np.max(np.abs(exp["z"]))) <= TOL64, call
        assert _rel(got["hu"], exp["hu"], qscale) <= TOL64, call
        if dim == 2:
            assert _rel(got["hv"], exp["hv"], qscale) <= TOL64, call
        assert abs(t - t_ref) <= TOL64 * t_ref, (call, t, t_ref)
    ref.close()


def test_noalloc_fp32_2d_matches_regular_entry_points_twice():
    """The FP32 state in 2D: the no-allocation call runs the fused stencil of
    the regular FP32 handle with the same launch shape, so both give the
    same state to FP32 rounding, on two calls in a row."""
    import torch

    w = W.antidune2d(nx=200, ny=96, seed=3)
    p = w["params"]
    cfg = sve.config_from_params(p, "fp32")
    names = ("h", "hu", "hv", "z")
    dev = {k: torch.tensor(np.asarray(w[k]), dtype=torch.float32, device="cuda").contiguous() for k in names}
    ref = sve.Solver(p, "fp32")
    ref.set_state(*(np.asarray(w[k], np.float32) for k in names))
    t = 0.0
    for call, n in enumerate((30, 17)):
        rc, t = sve.sve_step_noalloc(cfg, *(dev[k].data_ptr() for k in names), n, t)
        assert rc == sve.SVE_OK, sve.sve_strerror(rc)
        t_ref = ref.step(n)
        exp = ref.get_state()
        qscale = max(np.max(np.abs(exp["hu"])), np.max(np.abs(exp["hv"])))
        for k in names:
            scale = qscale if k in ("hu", "hv") else max(np.max(np.abs(exp[k])), 1e-12)
            assert _rel(dev[k].cpu().numpy(), exp[k], scale) <= 1e-6, (call, k)
        assert abs(t - t_ref) <= 1e-12 * t_ref, (call, t, t_ref)
    ref.close()


def test_noalloc_bad_input_leaves_arrays_untouched():
    """A non-finite input is reported by the device checks before any step,
    and the caller's arrays and time keep their values."""
    import torch

    w = W.dune2d(nx=64, ny=32, seed=2, lx=64.0, ly=32.0)
    cfg = sve.config_from_params(w["params"], "fp64")
    dev = {k: torch.tensor(w[k], dtype=torch.float64, device="cuda") for k in ("h", "hu", "hv", "z")}
    dev["hu"][5, 7] = float("nan")
    before = {k: v.clone() for k, v in dev.items()}
    rc, t = sve.sve_step_noalloc(cfg, dev["h"].data_ptr(), dev["hu"].data_ptr(), dev["hv"].data_ptr(),
                                 dev["z"].data_ptr(), 5, 1.5)
    assert rc == sve.SVE_ERR_NAN, sve.sve_strerror(rc)
    assert t == 1.5
    for k in ("h", "hv", "z"):
        assert torch.equal(before[k], dev[k]), k
    assert torch.equal(torch.isnan(before["hu"]), torch.isnan(dev["hu"]))


def test_noalloc_rejects_grid_beyond_scratch():
    import torch

    w = W.dune2d(nx=400, ny=300, seed=1, lx=400.0, ly=300.0)
    cfg = sve.config_from_params(w["params"], "fp64")
    dev = {k: torch.tensor(w[k], dtype=torch.float64, device="cuda") for k in ("h", "hu", "hv", "z")}
    before = dev["h"].clone()
    rc, t = sve.sve_step_noalloc(cfg, dev["h"].data_ptr(), dev["hu"].data_ptr(), dev["hv"].data_ptr(),
                                 dev["z"].data_ptr(), 3, 0.0)
    assert rc == sve.SVE_ERR_NOALLOC_SIZE
    assert "static scratch" in sve.sve_strerror(rc)
    assert torch.equal(before, dev["h"]) and t == 0.0
