"""The oracle on all host cores (``oracle.banded``: row bands of the
domain-decomposition API on threads) equals the single-threaded oracle run
bit for bit: states and time steps, for every ghost rule on the band edges
(inflow / free / wall, periodic in x, periodic in y) and for band counts that
leave bands of one row and of unequal heights."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle.banded import BandedRun
from paper_1307_0491_gb300 import workloads as W


def _case(name):
    if name == "dune_inflow":
        return W.dune2d(nx=40, ny=23, seed=41, lx=40.0, ly=23.0)
    if name == "x_periodic":
        return W.random_smooth(36, 17, seed=42, bc=("periodic", "periodic", "wall", "free"), A_g=0.05,
                               friction="strickler", K_st=30.0)
    if name == "y_periodic":
        return W.random_smooth(30, 19, seed=43, bc=("free", "wall", "periodic", "periodic"), A_g=0.02,
                               friction="darcy", f_dw=0.03)
    return W.antidune2d(nx=44, ny=21, seed=44)


@pytest.mark.parametrize("case", ["dune_inflow", "x_periodic", "y_periodic", "antidune_mpm"])
@pytest.mark.parametrize("nbands", [1, 3, 8])
def test_banded_oracle_equals_single_thread(case, nbands):
    w = _case(case)
    P = oracle.Params.from_workload(w["params"])
    nsteps = 15
    ref = oracle.get().run(P, nsteps, w["h"], w["hu"], w["hv"], w["z"])
    with BandedRun(oracle.get(), P, w["h"], w["hu"], w["hv"], w["z"], nbands=nbands, threads=4) as b:
        b.step(nsteps)
        got = b.state()
        assert np.array_equal(np.array(b.dts), ref["dts"])
        assert b.t == ref["t"]
    for k in ("h", "hu", "hv", "z"):
        assert np.array_equal(got[k], ref[k]), k


def test_banded_oracle_one_row_bands():
    w = W.dune2d(nx=16, ny=5, seed=45, lx=16.0, ly=5.0)
    P = oracle.Params.from_workload(w["params"])
    ref = oracle.get().run(P, 10, w["h"], w["hu"], w["hv"], w["z"])
    with BandedRun(oracle.get(), P, w["h"], w["hu"], w["hv"], w["z"], nbands=5, threads=5) as b:
        assert [y1 - y0 for y0, y1 in b.rows] == [1] * 5
        b.step(10)
        got = b.state()
    for k in ("h", "hu", "hv", "z"):
        assert np.array_equal(got[k], ref[k]), k


def test_banded_oracle_rejects_1d():
    w = W.dune1d(nx=32)
    P = oracle.Params.from_workload(w["params"])
    with pytest.raises(ValueError):
        BandedRun(oracle.get(), P, w["h"], w["hu"], w.get("hv"), w["z"])
