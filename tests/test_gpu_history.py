"""The per-step history ring (sve_set_history / sve_get_history): after
every step a record (t, dt, mass_h, mass_z, Sx, Sy) in device memory; the
last records of a run against the oracle's per-step time steps and mass
sums, through the CUDA graphs and the ring's wrap; the FP32 2D state (whose
calls of several steps then run one step at a time); 1D."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()


@pytest.mark.parametrize("dim", [2, 1])
def test_history_against_oracle(dim):
    if dim == 2:
        w = W.random_smooth(70, 33, seed=71, bc=("inflow_q", "free", "wall", "free"), A_g=0.02, q_in=0.3,
                            friction="strickler", K_st=40.0)
    else:
        w = W.dune1d(nx=300)
    n, cap = 37, 10
    s = sve.Solver(w["params"], "fp64")
    s.set_history(cap)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(n)  # graphs of 16 steps and single steps; the ring wraps
    rec = s.history(100)
    d = s.diag()
    s.close()
    ref = oracle.get().run(oracle.Params.from_workload(w["params"]), n, w["h"], w["hu"], w["hv"], w["z"])
    assert rec.shape == (cap, 6)
    t_ref = np.cumsum(ref["dts"])[-cap:]
    assert np.allclose(rec[:, 0], t_ref, rtol=1e-12, atol=0)
    assert np.allclose(rec[:, 1], ref["dts"][-cap:], rtol=1e-10, atol=0)
    assert np.allclose(rec[:, 2], ref["diag"][-cap:, 0], rtol=1e-11, atol=0)
    assert np.allclose(rec[:, 3], ref["diag"][-cap:, 1], rtol=1e-11, atol=0)
    assert np.all(rec[:, 4] > 0) and (np.all(rec[:, 5] > 0) if dim == 2 else np.all(rec[:, 5] == 0))
    assert rec[-1, 0] == d["t"] and rec[-1, 2] == d["mass_h"] and rec[-1, 3] == d["mass_z"]


def test_history_fp32_2d_and_switching():
    w = W.antidune2d(nx=120, ny=44, seed=72)
    s = sve.Solver(w["params"], "fp32")
    with pytest.raises(sve.SveError):
        s.history(5)  # off
    s.set_history(64)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(30)
    rec = s.history(64)
    dts = s.dts(30)
    assert rec.shape == (30, 6)
    assert np.array_equal(rec[:, 1], dts)
    assert np.allclose(rec[:, 0], np.cumsum(dts), rtol=1e-12)
    d = s.diag()
    assert rec[-1, 2] == d["mass_h"] and rec[-1, 3] == d["mass_z"]
    # the same run without the history: the same state (one step at a time
    # against the carried update: bit for bit)
    st = s.get_state()
    s.set_history(0)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(30)
    st2 = s.get_state()
    s.close()
    for k in ("h", "hu", "hv", "z"):
        assert np.array_equal(st[k], st2[k]), k
