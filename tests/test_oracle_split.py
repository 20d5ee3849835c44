"""Pins of the oracle's splitting scheme (orc_split_run; reading R13 of
oracle/sve_oracle.c): the alternative the paper's Sec. 2 contrasts with its
coupled method -- a shallow-water step, then the Exner equation updates the
bed.  Each test checks it against what the paper or the mathematics fix:
A_g = 0 leaves the bed rigid (Sec. 2) and the flow that of the coupled step;
the Exner update in flux form conserves the sediment on closed and periodic
grids and passes none through a wall; one step restated by hand on a small
grid (upwind side, dt/dx factor, the new flow's velocities); a uniform flow
moves no bed."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import workloads as W


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


def _run(orc, w, n, split, dts=None):
    P = oracle.Params.from_workload(w["params"])
    return orc.run(P, n, w["h"], w["hu"], w["hv"], w["z"], dts=dts, split=split)


def test_without_transport_the_bed_is_rigid_and_the_flow_that_of_the_coupled_step(orc):
    """A_g = 0: the splitting scheme's bed stays exactly where it was (Sec. 2:
    no transport, a rigid bed) and its first step's flow is the coupled
    step's.  (The coupled relaxation step itself moves a non-flat bed by a
    little even then -- its b-waves carry bed jumps at speeds b floored at
    beta_min a0 -- so after the first step the two flows part.)"""
    w = W.random_smooth(30, 14, seed=41, A_g=0.0, m_g=3.0, bc=("inflow_q", "free", "wall", "free"), q_in=0.4,
                        friction="strickler", K_st=40.0)
    a = _run(orc, w, 1, split=True)
    b = _run(orc, w, 1, split=False)
    for k in ("h", "hu", "hv"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["dts"], b["dts"])
    assert np.array_equal(_run(orc, w, 25, split=True)["z"], np.asarray(w["z"], dtype=np.float64))


@pytest.mark.parametrize("dim,bc", [
    (2, ("periodic", "periodic", "periodic", "periodic")),
    (2, ("wall", "wall", "wall", "wall")),
    (1, ("periodic", "periodic", "periodic", "periodic")),
    (1, ("wall", "wall", "wall", "wall")),
])
def test_exner_conserves_the_sediment(orc, dim, bc):
    w = W.random_smooth(48, 20 if dim == 2 else 1, seed=43, dim=dim, bc=bc, A_g=0.02, m_g=3.0)
    r = _run(orc, w, 60, split=True)
    z0 = float(np.sum(np.asarray(w["z"], dtype=np.float64)))
    assert abs(float(np.sum(r["z"])) - z0) <= 1e-13 * abs(z0)
    assert np.max(np.abs(r["z"] - w["z"])) > 1e-6  # the bed moved


def test_one_step_by_hand(orc):
    """Six periodic cells, velocities of both signs: the flow of one split
    step is the coupled step's without transport (same fixed dt), and the
    bed follows z_i - dt/dx (F_{i+1/2} - F_{i-1/2}) with F the Grass flux
    A_g u |u|^(m-1) of the new flow's upwind cell."""
    nx, L, A, m, dt = 6, 60.0, 0.03, 3.0, 0.05
    p = W.base_params(dim=1, nx=nx, ny=1, lx=L, ly=1.0, A_g=A, m_g=m,
                      bc=("periodic", "periodic", "periodic", "periodic"))
    h = np.array([1.0, 1.2, 0.9, 1.1, 1.05, 0.95])
    hu = np.array([0.5, 0.3, -0.2, -0.4, 0.1, 0.6])
    z = np.array([0.1, 0.15, 0.12, 0.08, 0.11, 0.09])
    w = {"params": p, "h": h, "hu": hu, "hv": None, "z": z}
    split = _run(orc, w, 1, split=True, dts=[dt])
    sw = _run(orc, dict(w, params=dict(p, A_g=0.0)), 1, split=False, dts=[dt])
    assert np.array_equal(split["h"], sw["h"]) and np.array_equal(split["hu"], sw["hu"])
    u = sw["hu"] / sw["h"]
    q = A * u * np.abs(u) ** (m - 1.0)
    F = np.empty(nx)  # F[i] at i + 1/2
    for i in range(nx):
        r = (i + 1) % nx
        s = u[i] + u[r]
        F[i] = q[i] if s > 0 else (q[r] if s < 0 else 0.5 * (q[i] + q[r]))
    expect = z - dt / (L / nx) * (F - np.roll(F, 1))
    assert np.max(np.abs(split["z"] - expect)) <= 1e-15 * np.max(np.abs(z)) * 10
    assert np.any(u < 0) and np.any(u > 0)


def test_uniform_flow_moves_no_bed(orc):
    nx, ny = 20, 8
    p = W.base_params(dim=2, nx=nx, ny=ny, lx=20.0, ly=8.0, A_g=0.05, m_g=3.0,
                      bc=("periodic", "periodic", "periodic", "periodic"))
    z = np.full((ny, nx), 0.3)
    w = {"params": p, "h": np.full((ny, nx), 2.0), "hu": np.full((ny, nx), 1.5), "hv": np.full((ny, nx), -0.4),
         "z": z}
    r = _run(orc, w, 10, split=True)
    assert np.array_equal(r["z"], z)
