"""Launch shape of the two-kernel step (sve_set_block_size: one-warp blocks
that spread a small grid's FP64 work over many SMs, or 256-thread blocks):
both against each other and the FP64 oracle, the automatic choice, and the
1D antidune test of Sec. 5.2 at the paper's resolution (J = 2400) to
T = 50 s."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
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


def rel(got, ref, scale=None):
    s = scale if scale is not None else max(float(np.max(np.abs(ref))), 1e-300)
    return float(np.max(np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))) / s)


def run(w, nsteps, block_size, precision="fp64", dts=None, persistent=0):
    s = sve.Solver(w["params"], precision)
    s.set_block_size(block_size)
    s.set_persistent(persistent)
    assert s.block_size == block_size
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if dts is None:
        s.step(nsteps)
    else:
        s.step_dt(dts)
    out = s.get_state()
    out["dts"] = s.dts(nsteps)
    out["diag"] = s.diag()
    out["launches"] = s.launches()
    out["counters"] = s.counters()
    s.close()
    return out


def orc_run(w, nsteps, dts=None):
    return oracle.get().run(oracle.Params.from_workload(w["params"]), nsteps, w["h"], w["hu"], w["hv"], w["z"],
                            dts=dts)


def parity(got, ref, dim, tol=TOL64, ctx=""):
    errs = {"h": rel(got["h"], ref["h"]), "hu": rel(got["hu"], ref["hu"]), "z": rel(got["z"], ref["z"])}
    if dim == 2:
        errs["hv"] = rel(got["hv"], ref["hv"], max(float(np.max(np.abs(ref["hu"]))), 1e-12))
    assert max(errs.values()) <= tol, (ctx, errs)
    return errs


def test_automatic_block_size():
    # 1001 interfaces: one warp per block; 1024 x 512: 128 threads
    s = sve.Solver(W.dune1d()["params"], "fp64")
    assert s.block_size == 32
    s.set_block_size(256)
    assert s.block_size == 256
    s.set_block_size(0)
    assert s.block_size == 32
    with pytest.raises(sve.SveError) as e:
        s.set_block_size(64)
    assert e.value.code == sve.SVE_ERR_ARG
    s.close()
    s = sve.Solver(W.dune2d()["params"], "fp64")
    assert s.block_size == 128
    s.close()


@pytest.mark.parametrize("w,n", [
    (W.dune1d(nx=1000), 600),
    (dict(W.dune1d(nx=777), params=dict(W.dune1d(nx=777)["params"], bc=("inflow_q", "free", "free", "free"),
                                         friction="strickler", K_st=40.0, q_in=0.5)), 600),
    (W.dune2d(nx=97, ny=45, lx=97.0, ly=45.0), 200),
    (W.dune2d(nx=300, ny=131, lx=300.0, ly=131.0), 100),
])
def test_block_sizes_match_oracle_and_each_other(w, n):
    dim = w["params"]["dim"]
    a = run(w, n, 32)
    b = run(w, n, 256)
    c = run(w, n, 128)
    ref = orc_run(w, n)
    parity(a, ref, dim, ctx="32")
    parity(b, ref, dim, ctx="256")
    parity(c, ref, dim, ctx="128")
    assert rel(c["dts"], b["dts"]) <= 1e-13
    # the same per-item code: identical time steps, states to round-off
    assert rel(a["dts"], b["dts"]) <= 1e-13
    for k in ("h", "hu", "z"):
        assert rel(a[k], b[k]) <= 1e-12, k
    assert a["launches"] == b["launches"] == 2 * n
    assert a["counters"]["steps"] == b["counters"]["steps"] == n
    # the persistent step where the grid is eligible (small)
    d = run(w, n, 32, persistent=1)
    parity(d, ref, dim, ctx="automatic")
    assert rel(d["dts"], b["dts"]) <= 1e-13
    assert d["counters"]["steps"] == n
    small = w["params"]["nx"] * w["params"]["ny"] <= 5000
    assert d["launches"] == (1 if small else 2 * n), d["launches"]
    ia, ib = a["counters"]["newton_iters"], b["counters"]["newton_iters"]
    assert abs(ia - ib) <= 1e-3 * ib + 2, (ia, ib)
    assert abs(a["diag"]["mass_h"] - b["diag"]["mass_h"]) <= 1e-13 * abs(b["diag"]["mass_h"])
    assert abs(a["diag"]["mass_z"] - b["diag"]["mass_z"]) <= 1e-13 * abs(b["diag"]["mass_z"])


def test_block_size_change_between_calls():
    """Switching the launch shape between calls (the captured graphs are
    rebuilt) continues the same run."""
    w = W.dune1d(nx=500)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    for bs in (32, 256, 128, 32):
        s.set_block_size(bs)
        s.step(40)
    got = s.get_state()
    s.close()
    parity(got, orc_run(w, 160), 1, ctx="switching")


def test_narrow_blocks_fp32_state():
    w = W.dune1d(nx=1000)
    a = run(w, 500, 32, precision="fp32")
    b = run(w, 500, 256, precision="fp32")
    ref = orc_run(w, 500)
    for k in ("h", "z"):
        assert rel(a[k], b[k]) <= 1e-5, k
        assert rel(a[k], ref[k]) <= 1e-4, k
    assert rel(a["hu"], ref["hu"]) <= 1e-3


def test_paper_antidune1d_full_resolution_T50():
    """Sec. 5.2 at the paper's resolution: J = 2400 cells on 24 m, Grass
    A_g = 1e-3, supercritical inflow, to T = 50 s (reading R10: 5 cm bump,
    for which the supercritical Bernoulli profile exists).  FP64 parity with
    the oracle over the whole run (~3e4 steps); the bump migrates upstream."""
    w = W.paper_antidune1d(nx=2400, bump=0.05, A_g=1e-3)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(40000)
    dts = s.dts(40000)
    s.close()
    n = int(np.searchsorted(np.cumsum(dts), 50.0)) + 1
    assert 1000 < n < 40000
    got = run(w, n, 32)
    ref = orc_run(w, n)
    assert ref["t"] >= 50.0
    parity(got, ref, 1, ctx="antidune T=50")
    assert abs(got["diag"]["t"] - ref["t"]) <= 1e-10 * ref["t"]
    x = (np.arange(2400) + 0.5) * 0.01

    def centroid(z):
        dz = np.clip(z - np.min(z), 0.0, None)
        return float(np.sum(x * dz) / np.sum(dz))

    assert centroid(got["z"]) < centroid(w["z"])  # upstream
