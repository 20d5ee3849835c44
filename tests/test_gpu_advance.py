"""sve_advance (state in, nsteps CFL steps, state out in one call) through
the C ABI: with page-locked host buffers (written by the last step's cell
update in the two-kernel step, copied after the FP32 2D step), pageable host
buffers (copied after the steps), device buffers and
in == out, in FP64 and in the FP32 state (fused 2D stencil and the 1D
kernels), for step counts that use the step graphs and a final single step.
Each result equals set_state + step + get_state bit for bit (the same
kernels in the same order), and the FP64 one the oracle at 1e-10."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu
KEYS = ("h", "hu", "hv", "z")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()


def reference(w, n, precision):
    s = sve.Solver(w["params"], precision)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = s.step(n)
    out = s.get_state()
    s.close()
    return out, t


def buffers(w, dtype, kind):
    import torch

    keys = [k for k in KEYS if w[k] is not None]
    src = {k: np.ascontiguousarray(w[k], dtype=dtype) for k in keys}
    if kind == "pinned":
        inp = {k: torch.from_numpy(src[k]).pin_memory().numpy() for k in keys}
        out = {k: torch.empty(src[k].shape, dtype=torch.from_numpy(src[k]).dtype).pin_memory().numpy()
               for k in keys}
    elif kind == "pageable":
        inp = src
        out = {k: np.empty_like(src[k]) for k in keys}
    else:
        inp = {k: torch.from_numpy(src[k]).cuda() for k in keys}
        out = {k: torch.empty_like(inp[k]) for k in keys}
    return inp, out


def host(a):
    return a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)


@pytest.mark.parametrize("kind", ["pinned", "pageable", "device"])
@pytest.mark.parametrize("n", [1, 37])
def test_advance_fp64_2d(kind, n):
    w = W.dune2d(nx=200, ny=77, seed=11, lx=200.0, ly=77.0)
    ref, t_ref = reference(w, n, "fp64")
    s = sve.Solver(w["params"], "fp64")
    inp, out = buffers(w, np.float64, kind)
    t = s.advance(n, inp, out)
    s.close()
    for k in KEYS:
        assert np.array_equal(host(out[k]), ref[k]), k
    assert t == t_ref
    orc = oracle.get().run(oracle.Params.from_workload(w["params"]), n, w["h"], w["hu"], w["hv"], w["z"])
    qs = max(np.max(np.abs(orc["hu"])), np.max(np.abs(orc["hv"])))
    assert np.max(np.abs(host(out["h"]) - orc["h"])) / np.max(orc["h"]) <= 1e-10
    assert np.max(np.abs(host(out["hu"]) - orc["hu"])) / qs <= 1e-10
    assert np.max(np.abs(host(out["z"]) - orc["z"])) / np.max(orc["z"]) <= 1e-10


def test_advance_in_place_pinned_and_repeated():
    w = W.dune2d(nx=96, ny=64, seed=12, lx=96.0, ly=64.0)
    ref, _ = reference(w, 40, "fp64")
    s = sve.Solver(w["params"], "fp64")
    buf, _ = buffers(w, np.float64, "pinned")
    s.advance(20, buf, buf)      # out == in
    s.advance(20, buf, buf)      # again from the result
    s.close()
    # two calls of 20 steps: the second restarts t at 0 but steps the same states
    for k in KEYS:
        assert np.array_equal(buf[k], ref[k]), k


@pytest.mark.parametrize("kind", ["pinned", "pageable", "device"])
@pytest.mark.parametrize("n", [1, 2, 21])
def test_advance_fp32_fused_2d(kind, n):
    """The FP32 2D step through sve_advance: one step, and calls of several
    steps (the carried update; device outputs written by the call's final
    update pass itself), equal to sve_step's result bit for bit."""
    w = W.antidune2d(nx=100, ny=44, seed=13)
    ref, t_ref = reference(w, n, "fp32")
    s = sve.Solver(w["params"], "fp32")
    inp, out = buffers(w, np.float32, kind)
    t = s.advance(n, inp, out)
    s.close()
    for k in KEYS:
        assert np.array_equal(host(out[k]), ref[k]), k
    assert t == t_ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_advance_1d_pinned(precision):
    w = W.dune1d(nx=300)
    dt = np.float64 if precision == "fp64" else np.float32
    ref, t_ref = reference(w, 50, precision)
    s = sve.Solver(w["params"], precision)
    inp, out = buffers(w, dt, "pinned")
    t = s.advance(50, inp, out)
    s.close()
    for k in ("h", "hu", "z"):
        assert np.array_equal(out[k], ref[k]), k
    assert t == t_ref


def test_advance_errors():
    w = W.dune2d(nx=64, ny=32, seed=14, lx=64.0, ly=32.0)
    s = sve.Solver(w["params"], "fp64")
    inp, out = buffers(w, np.float64, "pinned")
    keys = [inp[k].ctypes.data for k in KEYS]
    okeys = [out[k].ctypes.data for k in KEYS]
    rc, _ = sve.sve_advance(s.h, 0, keys, okeys, sve.SVE_HOST)
    assert rc == sve.SVE_ERR_ARG
    rc, _ = sve.sve_advance(s.h, 3, keys, okeys, 7)
    assert rc == sve.SVE_ERR_ARG
    rc, _ = sve.sve_advance(s.h, 3, keys, [okeys[0], okeys[1], None, okeys[3]], sve.SVE_HOST)
    assert rc == sve.SVE_ERR_ARG
    inp["h"][5, 7] = np.nan
    rc, _ = sve.sve_advance(s.h, 3, keys, okeys, sve.SVE_HOST)
    assert rc == sve.SVE_ERR_NAN
    # the handle steps on after a latched error once given a valid state
    inp["h"][5, 7] = 1.5
    rc, _ = sve.sve_advance(s.h, 3, keys, okeys, sve.SVE_HOST)
    assert rc == 0
    s.close()
