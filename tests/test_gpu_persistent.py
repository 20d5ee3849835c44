"""The persistent step of small grids (one cooperative launch of one-warp
blocks for up to 4096 steps, grid-wide barriers between the interface and
cell phases) against the two-kernel step from CUDA graphs: states, time
steps and simulated time equal up to round-off (the same per-interface and
per-cell functions, each kernel compiled on its own), for the 1D dune (5000 steps), the 1D antidune of
Sec. 5.2, 2D grids under every boundary rule with both transport laws and
frictions, fixed time steps and the FP32 state in 1D; the FP64 results also
against the oracle at 1e-10.  The bounded barrier wait: a launch whose
barrier can never open ends with SVE_ERR_SYNC and the handle steps on."""
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


def run(w, n, persistent, precision="fp64", dts=None):
    s = sve.Solver(w["params"], precision)
    s.set_block_size(32)
    s.set_persistent(1 if persistent else 0)
    used = s.persistent()
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if dts is None:
        t = s.step(n)
    else:
        s.step_dt(dts)
        t = float(np.sum(dts))
    out = s.get_state()
    out["t"] = t
    out["dts"] = s.dts(n)
    out["launches"] = s.launches()
    out["used"] = used
    out["diag"] = s.diag()
    s.close()
    return out


def assert_same(a, b, dim, tol=1e-12):
    """Equal up to round-off: the per-interface and per-cell functions are
    the same, but each kernel is compiled on its own, and the compiler may
    contract a multiply-add differently in each (no other difference)."""
    errs = {}
    for k in KEYS:
        if k == "hv" and dim == 1:
            continue
        scale = max(np.max(np.abs(b[k])), 1e-12)
        errs[k] = float(np.max(np.abs(np.asarray(a[k], np.float64) - b[k])) / scale)
    errs["dts"] = float(np.max(np.abs(a["dts"] - b["dts"]) / b["dts"]))
    errs["t"] = abs(a["t"] - b["t"]) / b["t"]
    assert max(errs.values()) <= tol, errs


def assert_oracle(got, w, n, dts=None):
    ref = oracle.get().run(oracle.Params.from_workload(w["params"]), n, w["h"], w["hu"], w["hv"], w["z"], dts=dts)
    for k in KEYS:
        if got[k] is None or w[k] is None:
            continue
        scale = max(np.max(np.abs(ref[k])), 1e-12) if k in ("h", "z") else max(
            np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])) if ref["hv"] is not None else 0.0, 1e-12)
        assert np.max(np.abs(got[k] - ref[k])) / scale <= 1e-10, k


def test_dune1d_full_config():
    w = W.dune1d()
    p = run(w, 5000, True)
    r = run(w, 5000, False)
    assert p["used"] and not r["used"]
    assert p["launches"] == 2  # 4096 + 904 steps
    assert_same(p, r, 1)
    assert_oracle(p, w, 5000)
    # mass diagnostics: the same sums in another order
    assert abs(p["diag"]["mass_h"] - r["diag"]["mass_h"]) <= 1e-13 * abs(r["diag"]["mass_h"])


def test_paper_antidune1d():
    w = W.paper_antidune1d(nx=2400, bump=0.05)
    p = run(w, 3000, True)
    r = run(w, 3000, False)
    assert p["used"]
    assert_same(p, r, 1)


@pytest.mark.parametrize("case", ["inflow_free_wall", "periodic", "antidune_mpm", "shields_manning"])
def test_small_2d_grids(case):
    if case == "inflow_free_wall":
        w = W.dune2d(nx=64, ny=40, seed=21, lx=64.0, ly=40.0)
        w["params"].update(bc=("inflow_q", "free", "wall", "free"))
    elif case == "periodic":
        w = W.random_smooth(48, 20, seed=22, bc=("periodic",) * 4, A_g=0.02, friction="darcy", f_dw=0.03)
    elif case == "antidune_mpm":
        w = W.antidune2d(nx=50, ny=24, seed=23)
    else:
        w = W.antidune2d(nx=40, ny=30, seed=24)
        w["params"].update(bedload="nielsen", friction="strickler", K_st=30.0)
    p = run(w, 300, True)
    r = run(w, 300, False)
    assert p["used"]
    assert_same(p, r, 2)
    assert_oracle(p, w, 300)


def test_fixed_steps():
    w = W.dune2d(nx=40, ny=24, seed=25, lx=40.0, ly=24.0)
    dts = np.full(120, 0.05)
    p = run(w, 120, True, dts=dts)
    r = run(w, 120, False, dts=dts)
    assert_same(p, r, 2)
    assert_oracle(p, w, 120, dts=dts)


def test_fp32_state_1d():
    w = W.dune1d(nx=500)
    p = run(w, 1000, True, "fp32")
    r = run(w, 1000, False, "fp32")
    assert p["used"]
    assert_same(p, r, 1)


def test_large_grid_not_eligible():
    w = W.dune2d()
    s = sve.Solver(w["params"], "fp64")
    s.set_persistent(1)
    assert not s.persistent()
    s.close()


def test_bounded_barrier_wait():
    w = W.dune1d(nx=300)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    before = s.get_state()
    rc = sve.load().sve_check_sync_timeout(s.h, 20000)
    assert rc == sve.SVE_ERR_SYNC
    after = s.get_state()
    for k in ("h", "hu", "z"):
        assert np.array_equal(before[k], after[k]), k  # the step never reached its update
    # the context stays usable: a fresh state steps as usual
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(50)
    got = s.get_state()
    s.close()
    ref = run(w, 50, False)
    for k in ("h", "hu", "z"):
        assert np.array_equal(got[k], ref[k]), k


def test_persistent_then_host_mirror():
    """sve_advance with the persistent step: the steps before the last run
    persistent, the last one as the two-kernel step that stores into the
    page-locked host buffers."""
    import torch

    w = W.dune1d(nx=400)
    r = run(w, 60, False)
    s = sve.Solver(w["params"], "fp64")
    s.set_persistent(1)
    keys = ("h", "hu", "z")
    inp = {k: torch.from_numpy(np.ascontiguousarray(w[k], dtype=np.float64)).pin_memory().numpy() for k in keys}
    out = {k: torch.empty(np.shape(w[k]), dtype=torch.float64).pin_memory().numpy() for k in keys}
    t = s.advance(60, inp, out)
    assert s.launches() == 3  # one persistent launch, then the last step's two kernels
    s.close()
    errs = {k: float(np.max(np.abs(out[k] - r[k])) / np.max(np.abs(r[k]))) for k in keys}
    assert max(errs.values()) <= 1e-12, errs
    assert abs(t - r["t"]) <= 1e-12 * r["t"]
