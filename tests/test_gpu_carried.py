"""The FP32 2D state's carried update: within one call of n steps, the solve
pass of step k applies step k - 1's update as it reads the state (the
apply pass runs once, after the last step).  A call of n steps must equal
n calls of one step (solve pass + apply pass each) bit for bit -- states,
time steps, simulated time, mass sums -- under every boundary rule, with CFL
and with recorded time steps, for call lengths that end on either state
buffer and that include the graphs of 16 carried steps."""
from __future__ import annotations

import numpy as np
import pytest

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


CASES = [
    (97, 45, ("periodic", "periodic", "periodic", "periodic"), dict()),
    (65, 33, ("wall", "wall", "wall", "wall"), dict(friction="darcy", f_dw=0.03)),
    (33, 19, ("inflow_qh", "free", "wall", "free"), dict(q_in=0.9, h_in=1.9, friction="strickler", K_st=40.0)),
    (70, 37, ("inflow_q", "free", "periodic", "periodic"), dict(q_in=0.5, friction="strickler", K_st=30.0)),
    (40, 64, ("periodic", "periodic", "inflow_q", "free"), dict(q_in=0.4)),
]


def _run(w, n, one_at_a_time, dts=None):
    s = sve.Solver(w["params"], "fp32")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if dts is None:
        if one_at_a_time:
            logged = []
            for _ in range(n):
                s.step(1)
                logged.append(s.dts(1)[0])
            got_dts = np.array(logged)
        else:
            s.step(n)
            got_dts = s.dts(n)
    else:
        if one_at_a_time:
            for k in range(n):
                s.step_dt(dts[k:k + 1])
        else:
            s.step_dt(dts)
        got_dts = np.asarray(dts)
    out = s.get_state()
    out["dts"] = got_dts
    out["diag"] = s.diag()
    out["steps"] = s.counters()["steps"]
    s.close()
    return out


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("n", [1, 2, 17, 34])
def test_carried_call_equals_single_steps(case, n):
    nx, ny, bc, extra = CASES[case]
    w = W.random_smooth(nx, ny, seed=nx * ny + n, bc=bc, A_g=0.02, **extra)
    a = _run(w, n, one_at_a_time=False)
    b = _run(w, n, one_at_a_time=True)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (k, float(np.max(np.abs(a[k].astype(np.float64) - b[k]))))
    assert np.array_equal(a["dts"], b["dts"])
    assert a["diag"]["t"] == b["diag"]["t"]
    assert a["diag"]["mass_h"] == b["diag"]["mass_h"] and a["diag"]["mass_z"] == b["diag"]["mass_z"]
    assert a["steps"] == b["steps"] == n


def test_carried_call_with_recorded_steps():
    nx, ny, bc, extra = CASES[3]
    w = W.random_smooth(nx, ny, seed=5, bc=bc, A_g=0.02, **extra)
    dts = np.linspace(0.02, 0.05, 35)
    a = _run(w, 35, one_at_a_time=False, dts=dts)
    b = _run(w, 35, one_at_a_time=True, dts=dts)
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), k
    assert a["diag"]["t"] == b["diag"]["t"]


def test_carried_call_latches_a_bad_step():
    """A recorded step far above the CFL limit inside a carried call latches
    a state error (no trap); the handle stays usable after a new state."""
    nx, ny, bc, extra = CASES[1]
    w = W.random_smooth(nx, ny, seed=9, bc=bc, A_g=0.02, **extra)
    s = sve.Solver(w["params"], "fp32")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    dts = np.full(20, 0.02)
    dts[7] = 50.0
    with pytest.raises(sve.SveError):
        s.step_dt(dts)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(5)
    assert np.all(np.isfinite(s.get_state()["h"]))
    s.close()
