"""The splitting scheme on the GPU (sve_set_scheme(SVE_SCHEME_SPLIT); the
alternative Sec. 2 of the paper contrasts with its coupled method): against
the oracle's splitting scheme (reading R13 of oracle/sve_oracle.c) element
by element at 1e-10 after the config's step count, in 1D and 2D, under every
boundary rule and for the Grass and a Shields-parameter law; steps in CUDA
graphs equal single steps; switching the scheme re-projects the state."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu

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


def gpu_split(w, n, one_at_a_time=False):
    s = sve.Solver(w["params"], "fp64")
    s.set_scheme("split")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if one_at_a_time:
        for _ in range(n):
            s.step(1)
    else:
        s.step(n)
    out = s.get_state()
    out["diag"] = s.diag()
    s.close()
    return out


def rel(a, b, scale):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b))) / scale


CASES = {
    "dune1d_periodic": lambda: W.dune1d(nx=400),
    "antidune1d": lambda: W.paper_antidune1d(nx=600, bump=0.05),
    "walls2d_grass": lambda: W.random_smooth(60, 34, seed=61, bc=("wall", "wall", "wall", "wall"), A_g=0.02),
    "inflow2d_strickler": lambda: W.random_smooth(57, 31, seed=62, bc=("inflow_q", "free", "periodic", "periodic"),
                                                  A_g=0.02, q_in=0.4, friction="strickler", K_st=40.0),
    "inflowqh2d": lambda: W.random_smooth(40, 22, seed=63, bc=("inflow_qh", "free", "wall", "free"), A_g=0.01,
                                          q_in=0.9, h_in=1.9, friction="darcy", f_dw=0.03),
    "mpm_antidune2d": lambda: W.antidune2d(nx=96, ny=40, seed=64),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_split_matches_oracle(case):
    w = CASES[case]()
    n = 150
    got = gpu_split(w, n)
    P = oracle.Params.from_workload(w["params"])
    ref = oracle.get().run(P, n, w["h"], w["hu"], w["hv"], w["z"], split=True)
    qs = max(float(np.max(np.abs(ref["hu"]))), float(np.max(np.abs(ref["hv"]))) if ref["hv"] is not None else 0.0)
    assert rel(got["h"], ref["h"], float(np.max(ref["h"]))) <= 1e-10
    assert rel(got["hu"], ref["hu"], qs) <= 1e-10
    if ref["hv"] is not None:
        assert rel(got["hv"], ref["hv"], qs) <= 1e-10
    zscale = max(float(np.max(np.abs(ref["z"]))), float(np.max(ref["h"])))
    assert rel(got["z"], ref["z"], zscale) <= 1e-10
    assert got["diag"]["t"] == pytest.approx(ref["t"], rel=1e-12)
    assert got["diag"]["mass_z"] == pytest.approx(ref["diag"][-1][1], rel=1e-12)
    assert np.max(np.abs(ref["z"] - np.asarray(w["z"], dtype=np.float64))) > 1e-7  # the bed moved


def test_split_graphs_equal_single_steps():
    w = CASES["inflow2d_strickler"]()
    a = gpu_split(w, 40)
    b = gpu_split(w, 40, one_at_a_time=True)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert a["diag"] == b["diag"]


def test_switching_scheme_reprojects():
    """Setting the scheme after the state equals setting it before; back to
    the coupled step gives the coupled run."""
    w = CASES["walls2d_grass"]()
    ref = gpu_split(w, 20)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.set_scheme("split")
    assert s.scheme == "split"
    s.step(20)
    got = s.get_state()
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
    s.set_scheme("coupled")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(20)
    coupled = s.get_state()
    s.close()
    c = sve.Solver(w["params"], "fp64")
    c.set_state(w["h"], w["hu"], w["hv"], w["z"])
    c.step(20)
    for k in FIELDS:
        assert np.array_equal(coupled[k], c.get_state()[k]), k
    c.close()


def test_split_refused_where_unsupported():
    w = W.random_smooth(20, 10, seed=65, A_g=0.01)
    s = sve.Solver(w["params"], "fp32")
    with pytest.raises(sve.SveError):
        s.set_scheme("split")
    s.close()
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.set_scheme("split")
    with pytest.raises(sve.SveError):
        s.record_forward(5)
    s.close()
