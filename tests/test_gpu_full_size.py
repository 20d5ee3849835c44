"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (default launch shape of each grid, CUDA graphs, the batch's
autotuned schedule), against the FP64 oracle on all host cores (row bands of
its block API on threads, bit-identical to the single-threaded oracle):

* the 2D dune (1024 x 512) for its full 2000 steps, element by element;
* the 2D antidune (8192 x 4096, the largest grid) for 50 steps, element by
  element, in FP64, and the FP32 state's error after the same steps; a
  1024 x 512 crop of it for the config's full 1000 steps;
* the 256-run ensemble for its full 1000 steps, the smallest, the median and
  the largest run element by element;
* the adjoint config (2048 x 1024, periodic): the gradient against central
  differences of the GPU forward run (a property that holds at any size);
* the 2D bump of Sec. 5.3 on a 1000 x 1000 grid (the large-grid launch
  shape) for 200 steps, element by element, both A_g of the paper.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle.banded import BandedRun
from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
FIELDS = ("h", "hu", "hv", "z")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()


def oracle_banded(w, nsteps):
    P = oracle.Params.from_workload(w["params"])
    with BandedRun(oracle.get(), P, w["h"], w["hu"], w["hv"], w["z"]) as b:
        b.step(nsteps)
        out = b.state()
        out["t"] = b.t
        out["dts"] = np.array(b.dts)
    return out


def rel_errs(got, ref):
    qs = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])), 1e-12)
    scale = {"h": np.max(np.abs(ref["h"])), "z": max(np.max(np.abs(ref["z"])), 1e-12), "hu": qs, "hv": qs}
    return {k: float(np.max(np.abs(np.asarray(got[k], np.float64) - ref[k])) / scale[k]) for k in FIELDS}


def test_dune2d_full_config_2000_steps():
    w = W.dune2d()
    n = 2000
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = s.step(n)
    got = s.get_state()
    dts = s.dts(n)
    s.close()
    ref = oracle_banded(w, n)
    errs = rel_errs(got, ref)
    assert max(errs.values()) <= TOL64, errs
    assert np.max(np.abs(dts - ref["dts"]) / ref["dts"]) <= 1e-10
    assert abs(t - ref["t"]) <= 1e-10 * ref["t"]


def test_antidune2d_full_grid_steps_fp64_and_fp32():
    w = W.antidune2d()
    n = 50
    ref = oracle_banded(w, n)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(n)
    got = s.get_state()
    dts = s.dts(n)
    s.close()
    errs = rel_errs(got, ref)
    assert max(errs.values()) <= TOL64, errs
    assert np.max(np.abs(dts - ref["dts"]) / ref["dts"]) <= 1e-12
    del got
    # the FP32 state (fused stencil) against the same FP64 oracle result
    s = sve.Solver(w["params"], "fp32")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(n)
    got = s.get_state()
    s.close()
    e32 = rel_errs(got, ref)
    # the FP32 state's bound against the FP64 oracle (as on the smaller
    # grids; the relative errors of the discharges are taken against the
    # largest |hu|, |hv|)
    assert e32["h"] <= 1e-4 and e32["z"] <= 1e-4, e32
    assert e32["hu"] <= 1e-3 and e32["hv"] <= 1e-3, e32


def test_antidune_crop_full_step_count():
    """A 1024 x 512 crop of the antidune grid (same cells, the first 512
    rows and 1024 columns: 3 x 1.5 m) for the config's full 1000 steps."""
    full = W.antidune2d()
    w = {k: (np.ascontiguousarray(full[k][:512, :1024]) if k in FIELDS else full[k]) for k in full}
    w["params"] = dict(full["params"], nx=1024, ny=512, lx=3.0, ly=1.5)
    del full
    n = 1000
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = s.step(n)
    got = s.get_state()
    s.close()
    ref = oracle_banded(w, n)
    errs = rel_errs(got, ref)
    assert max(errs.values()) <= TOL64, errs
    assert abs(t - ref["t"]) <= 1e-10 * ref["t"]


def test_ensemble_full_size_sampled_runs():
    runs = W.ensemble()
    n = 1000
    b = sve.Batch([r["params"] for r in runs], "fp64")
    for i, r in enumerate(runs):
        b.set_state(i, r["h"], r["hu"], r["hv"], r["z"])
    b.autotune(2)
    b.step(n)
    cells = [r["params"]["nx"] * r["params"]["ny"] for r in runs]
    order = np.argsort(cells, kind="stable")
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    outs = {i: (b.get_state(i), b.diag(i)["t"]) for i in picks}
    b.close()
    for i in picks:
        got, t = outs[i]
        ref = oracle_banded(runs[i], n)
        errs = rel_errs(got, ref)
        assert max(errs.values()) <= TOL64, (i, errs)
        assert abs(t - ref["t"]) <= 1e-10 * ref["t"], i


def test_adjoint_config_full_grid_vs_central_differences():
    w = W.adjoint_dune()
    p = w["params"]
    nx, ny = p["nx"], p["ny"]
    # Smooth periodic ripples of 0.1 mm on the depth and 1e-4 m^2/s on the
    # discharge break the exact ties of neighbouring celerity maxima: with a
    # uniform discharge and m_g = 3 the bound g H^2 dQ/du_n of Eq. (ab) does
    # not depend on H, so both sides of every interface outside the bump
    # give the same b0 and the discrete map has a kink in m_g at 3 (the
    # one-sided derivatives differ by 3e-4 relative), which central
    # differences straddle.
    X = (np.arange(nx) + 0.5)[None, :] / nx
    Y = (np.arange(ny) + 0.5)[:, None] / ny
    w["h"] = w["h"] + 1e-4 * np.sin(2 * np.pi * (3 * X + 2 * Y)) * np.cos(2 * np.pi * 5 * X)
    w["hu"] = w["hu"] + 1e-4 * np.cos(2 * np.pi * (2 * X - 3 * Y) + 0.3)
    n = 20
    tgt = W.adjoint_dune(A_g=1.1e-3, m_g=3.1, K_st=36.0, shift=5.0)
    st = sve.Solver(tgt["params"], "fp64")
    st.set_state(tgt["h"], tgt["hu"], tgt["hv"], tgt["z"])
    st.step(n)
    z_target = st.get_state()["z"]
    st.close()

    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, 0)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - z_target))
    s.close()
    s2 = sve.Solver(p, "fp64")
    s2.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s2.step(n)
    dts = s2.dts(n)
    s2.close()

    def loss(pp, z0=None):
        f = sve.Solver(pp, "fp64")
        f.set_state(w["h"], w["hu"], w["hv"], w["z"] if z0 is None else z0)
        f.step_dt(dts)
        z = f.get_state()["z"]
        f.close()
        return float(np.sum((z - z_target) ** 2))

    for idx, name in enumerate(("A_g", "m_g", "K_st")):
        v = p[name]
        e = (1e-4 if name == "K_st" else 1e-6) * abs(v)
        pp, pm = dict(p), dict(p)
        pp[name] = v + e
        pm[name] = v - e
        fd = (loss(pp) - loss(pm)) / (2 * e)
        assert abs(gp[idx] - fd) <= 1e-5 * abs(fd) + 1e-9, (name, gp[idx], fd)
    d = np.sin(2 * np.pi * (2 * X + Y) + 0.7)
    e = 1e-6
    fd = (loss(p, w["z"] + e * d) - loss(p, w["z"] - e * d)) / (2 * e)
    ad = float(np.sum(grads["z"] * d))
    assert abs(ad - fd) <= 1e-5 * abs(fd) + 1e-9, (ad, fd)


@pytest.mark.parametrize("A_g", [1.0, 0.1])
def test_paper_bump2d_1000x1000(A_g):
    """The 2D bump of Sec. 5.3 (1000 x 1000 m, q0 = 10, h = 10 - z_b, 2D
    Grass m_g = 3, inflow upstream, free elsewhere) on a 1000 x 1000 grid --
    128-thread blocks, CUDA graphs: the large-grid launch of the paper's
    4000 x 4000 run -- for 200 steps, element by element at 1e-10 against
    the banded oracle, with every time step."""
    w = W.paper_bump2d(nx=1000, ny=1000, A_g=A_g)
    s = sve.Solver(w["params"], "fp64")
    assert s.block_size == 128
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = s.step(200)
    got = s.get_state()
    dts = s.dts(200)
    s.close()
    ref = oracle_banded(w, 200)
    errs = rel_errs(got, ref)
    assert max(errs.values()) <= TOL64, errs
    assert abs(t - ref["t"]) <= TOL64 * ref["t"]
    assert np.max(np.abs(dts - ref["dts"])) <= TOL64 * np.max(ref["dts"])
