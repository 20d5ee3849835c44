"""GPU parity (through the C ABI) on the method's edge cases, element by
element against the FP64 oracle at the FP64 bar (relative L-infinity 1e-10
per field after the run), with the device's safeguard counters
(sve_get_safeguards) proving that each branch ran on the GPU:

  * positivity stress (Sec. 3, positivity of the relaxation scheme): a dam
    break onto a 1 mm layer at CFL 0.5, 1D and a walled 2D channel;
  * the bed-jump bound of the celerities (the stronger bound Sec. 3 says
    well-definedness may need after Eq. ab; reading R1): flow over a bed
    step a third of the depth high, 1D and an oblique 2D step;
  * Newton step halving and the doubled celerity (readings R2, R12): two
    supercritical streams colliding in a walled channel, 1D and 2D, the
    launch shapes of small and large grids;
  * the walled 2D lake at rest (Sec. 4: the scheme is not well balanced):
    the spurious velocities the oracle develops, reproduced.
"""
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


def _rel(got, ref, scale):
    return float(np.max(np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))) / scale)


def _gpu(w, nsteps, precision="fp64", block_size=None):
    s = sve.Solver(w["params"], precision)
    if block_size is not None:
        s.set_block_size(block_size)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    t = s.step(nsteps)
    out = s.get_state()
    out["t"] = t
    out["dts"] = s.dts(nsteps)
    out["safeguards"] = s.safeguards()
    out["diag"] = s.diag()
    s.close()
    return out


def _orc(w, nsteps):
    return oracle.get().run(oracle.Params.from_workload(w["params"]), nsteps, w["h"], w["hu"], w["hv"], w["z"])


def _assert_parity(got, ref, dim, ctx):
    """Relative L-infinity error per field: depth against the largest depth,
    discharges against the largest discharge, bed elevation against the
    elevation scale of the flow, max(|z|, h) -- the beds here start flat
    (z = 0) and move by centimetres under a metre of water, so the bed's own
    range would measure rounding in metres of water against centimetres."""
    hs = np.max(np.abs(ref["h"]))
    qs = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])) if dim == 2 else 0.0, 1e-12)
    zs = max(np.max(np.abs(ref["z"])), hs)
    errs = {"h": _rel(got["h"], ref["h"], hs), "hu": _rel(got["hu"], ref["hu"], qs), "z": _rel(got["z"], ref["z"], zs)}
    if dim == 2:
        errs["hv"] = _rel(got["hv"], ref["hv"], qs)
    assert max(errs.values()) <= TOL64, f"{ctx}: {errs}"
    assert abs(got["t"] - ref["t"]) <= TOL64 * ref["t"], (ctx, got["t"], ref["t"])
    assert np.max(np.abs(got["dts"] - ref["dts"])) <= TOL64 * np.max(ref["dts"]), ctx
    return errs


def _thin_dam_break_2d(nx=120, ny=24, h_thin=1e-3):
    """The 1D positivity stress case extruded across a walled channel, with
    the dam line bent so that y-interfaces carry jumps as well."""
    w = W.thin_dam_break(nx, h_thin)
    L = w["params"]["lx"]
    ly = L * ny / nx
    x = (np.arange(nx) + 0.5) * (L / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    h = np.where(X < 0.5 * L + 0.3 * np.sin(2 * np.pi * Y / ly), 1.0, h_thin)
    p = W.base_params(dim=2, nx=nx, ny=ny, lx=L, ly=ly, A_g=1e-3, cfl=0.5, bc=("wall", "wall", "wall", "wall"))
    return dict(params=p, h=h, hu=np.zeros_like(h), hv=np.zeros_like(h), z=np.zeros_like(h), nsteps=None)


@pytest.mark.parametrize("dim", [1, 2])
def test_thin_dam_break_cfl05(dim):
    """Dam break from 1 m onto a 1 mm layer at CFL 0.5 with walls: the depth
    stays positive everywhere, water is conserved, and the state equals the
    oracle's after 400 steps (1D: to t ~ 0.9 s)."""
    w = W.thin_dam_break(200, 1e-3) if dim == 1 else _thin_dam_break_2d()
    n = 400 if dim == 1 else 250
    got = _gpu(w, n)
    ref = _orc(w, n)
    _assert_parity(got, ref, dim, f"thin dam break {dim}D")
    assert np.min(got["h"]) > 0.0
    cell = w["params"]["lx"] / w["params"]["nx"] * (w["params"]["ly"] / w["params"]["ny"] if dim == 2 else 1.0)
    m0 = float(np.sum(w["h"])) * cell
    assert abs(got["diag"]["mass_h"] - m0) <= 1e-13 * m0


@pytest.mark.parametrize("dim", [1, 2])
def test_bed_step_engages_the_bed_jump_bound(dim):
    """Flow over a bed step a third of the depth high: the celerity a is set
    by the bed-jump bound at the step (counted on the device), and the run
    equals the oracle's."""
    w = W.bed_step(100) if dim == 1 else W.bed_step(80, dim=2, ny=40)
    n = 300 if dim == 1 else 200
    got = _gpu(w, n)
    ref = _orc(w, n)
    _assert_parity(got, ref, dim, f"bed step {dim}D")
    assert got["safeguards"]["raised"] > 0, got["safeguards"]


@pytest.mark.parametrize("dim,block_size", [(1, None), (1, 128), (2, None), (2, 128)])
def test_colliding_streams_halve_and_double(dim, block_size):
    """Two supercritical streams (Froude 3) colliding at mid-channel: Newton
    steps are halved, a is doubled where R1's celerities admit no root, the
    bed-jump bound engages at the bed features the jump builds, near-dry
    cells appear at the walls -- and the state and every time step equal the
    oracle's after 300 steps, for the automatic launch shape and 128-thread
    blocks."""
    w = W.colliding_streams(200) if dim == 1 else W.colliding_streams(60, dim=2, ny=24, ymod=0.2)
    got = _gpu(w, 300, block_size=block_size)
    ref = _orc(w, 300)
    _assert_parity(got, ref, dim, f"colliding streams {dim}D block {block_size}")
    sg = got["safeguards"]
    assert sg["halvings"] > 0 and sg["retries"] > 0 and sg["raised"] > 0, sg
    assert np.min(got["h"]) > 0.0


def test_colliding_streams_fp32_state():
    """The FP32-state 2D step (fused stencil) on the colliding streams: it
    takes the same safeguards on its own solves, keeps every depth positive
    and conserves water to FP32 rounding."""
    w = W.colliding_streams(60, dim=2, ny=24, ymod=0.2)
    got = _gpu(w, 300, precision="fp32")
    sg = got["safeguards"]
    assert sg["halvings"] > 0 and sg["retries"] > 0, sg
    assert np.min(got["h"]) > 0.0 and np.all(np.isfinite(got["hu"]))
    cell = w["params"]["lx"] / 60 * w["params"]["ly"] / 24
    m0 = float(np.sum(w["h"])) * cell
    assert abs(got["diag"]["mass_h"] - m0) <= 1e-5 * m0


def test_walled_lake_at_rest_2d():
    """Water at rest over a bump in a walled basin (Sec. 4: the scheme is not
    well balanced): the GPU develops the oracle's spurious velocities, equal
    to it element by element, and conserves water."""
    w = W.lake_at_rest(64, dim=2, ny=32)
    got = _gpu(w, 400)
    ref = _orc(w, 400)
    _assert_parity(got, ref, 2, "lake at rest 2D")
    u = np.abs(got["hu"] / got["h"])
    assert np.max(u) > 1e-6  # not well balanced
    m0 = float(np.sum(w["h"])) * (10.0 / 64) * (5.0 / 32)
    assert abs(got["diag"]["mass_h"] - m0) <= 1e-13 * m0
