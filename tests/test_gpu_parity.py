"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

FP64: relative L-infinity error <= 1e-10 per field after the run's step count
(the bar of the FP64 path).  Sizes span several thread blocks with ragged
tails; every boundary type, both bedload laws and both friction laws are
exercised.  FP32 state: the error against the FP64 oracle is measured and
bounded (stated per case in the assertion)."""
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


def rel_err(got, ref, scale=None):
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    s = scale if scale is not None else max(np.max(np.abs(ref)), 1e-300)
    return float(np.max(np.abs(got - ref)) / s)


def run_gpu(w, nsteps, precision="fp64", dts=None, block_size=None, persistent=None):
    s = sve.Solver(w["params"], precision)
    if block_size is not None:
        s.set_block_size(block_size)
    if persistent is not None:
        s.set_persistent(persistent)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if dts is None:
        t = s.step(nsteps)
    else:
        s.step_dt(dts)
        t = float(np.sum(dts))
    out = s.get_state()
    out["t"] = t
    out["dts"] = s.dts(nsteps)
    out["diag"] = s.diag()
    out["launches"] = s.launches()
    s.close()
    return out


def run_orc(w, nsteps, dts=None):
    return oracle.get().run(oracle.Params.from_workload(w["params"]), nsteps, w["h"], w["hu"], w["hv"], w["z"],
                            dts=dts)


def assert_parity(got, ref, dim, tol=TOL64, ctx=""):
    qscale = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])) if dim == 2 else 0.0, 1e-12)
    errs = {"h": rel_err(got["h"], ref["h"]), "hu": rel_err(got["hu"], ref["hu"], qscale),
            "z": rel_err(got["z"], ref["z"])}
    if dim == 2:
        errs["hv"] = rel_err(got["hv"], ref["hv"], qscale)
    worst = max(errs.values())
    assert worst <= tol, f"{ctx} parity {errs}"
    return errs


@pytest.mark.parametrize("block_size,persistent,launches", [(32, 1, 2), (32, 0, 2 * 5000), (256, 0, 2 * 5000)])
def test_c1_dune1d_full(block_size, persistent, launches):
    """1D dune, N = 1000, periodic, 5000 CFL steps (the full 1D config): the
    persistent step (two cooperative launches of 4096 + 904 steps), and the
    two-kernel step with one-warp blocks (the automatic shape on this grid)
    and with 256-thread blocks."""
    w = W.dune1d()
    got = run_gpu(w, 5000, block_size=block_size, persistent=persistent)
    ref = run_orc(w, 5000)
    assert_parity(got, ref, 1, ctx=f"C1 block {block_size} persistent {persistent}")
    assert abs(got["t"] - ref["t"]) <= 1e-10 * ref["t"]
    assert np.max(np.abs(got["dts"] - ref["dts"])) <= 1e-10 * np.max(ref["dts"])
    assert got["launches"] == launches


@pytest.mark.parametrize("nx,ny,bc,extra", [
    (200, 77, ("inflow_q", "free", "free", "free"), dict(friction="strickler", K_st=40.0, q_in=0.5)),
    (131, 90, ("periodic", "periodic", "periodic", "periodic"), dict()),
    (97, 64, ("wall", "wall", "wall", "wall"), dict(friction="darcy", f_dw=0.03)),
    (64, 129, ("inflow_qh", "free", "wall", "free"), dict(q_in=0.9, h_in=1.9)),
])
def test_2d_dune_small_grids(nx, ny, bc, extra):
    """2D Grass dune, several blocks plus ragged tails, each boundary rule,
    300 CFL steps."""
    w = W.dune2d(nx=nx, ny=ny, seed=nx + ny, lx=1000.0 * nx / 1024, ly=500.0 * ny / 512)
    w["params"].update(bc=bc, **extra)
    got = run_gpu(w, 300)
    ref = run_orc(w, 300)
    assert_parity(got, ref, 2, ctx=f"{nx}x{ny} {bc}")
    assert abs(got["t"] - ref["t"]) <= 1e-10 * ref["t"]


@pytest.mark.parametrize("m_g", [1.0, 2.0, 4.0, 2.5])
def test_2d_grass_exponents(m_g):
    """Every Grass exponent path (integer powers and pow)."""
    w = W.dune2d(nx=80, ny=48, seed=5, lx=80.0, ly=48.0, A_g=5e-3, m_g=m_g)
    got = run_gpu(w, 200)
    ref = run_orc(w, 200)
    assert_parity(got, ref, 2, ctx=f"m_g={m_g}")


def test_c2_dune2d_full_grid_first_steps():
    """The full 2D dune grid (1024 x 512, Grass + Strickler, inflow/free),
    10 CFL steps against the oracle element by element."""
    w = W.dune2d()
    got = run_gpu(w, 10)
    ref = run_orc(w, 10)
    assert_parity(got, ref, 2, ctx="C2 10 steps")


def test_c2_physics_long_run_reduced_grid():
    """C2 physics on a 128 x 64 grid for the config's 2000 steps."""
    w = W.dune2d(nx=128, ny=64, seed=0, lx=1000.0, ly=500.0)
    got = run_gpu(w, 2000)
    ref = run_orc(w, 2000)
    assert_parity(got, ref, 2, ctx="C2 physics 2000 steps")


def test_c3_antidune_mpm_darcy_reduced_grid():
    """Antidune physics (MPM + Darcy, supercritical inflow, random bed) on a
    384 x 192 grid, 100 steps."""
    w = W.antidune2d(nx=384, ny=192, seed=0)
    got = run_gpu(w, 100)
    ref = run_orc(w, 100)
    assert_parity(got, ref, 2, ctx="C3 physics")


@pytest.mark.parametrize("law,fric", [("flvb", "darcy"), ("nielsen", "darcy"), ("ribberink", "darcy"),
                                      ("camenen", "darcy"), ("camenen", "strickler"), ("ribberink", "strickler")])
def test_shields_laws_2d(law, fric):
    """The other transport laws of Sec. 2 (Eqs. FLVB, Nielsen, Ribberink,
    Camenen) on the antidune physics (supercritical inflow, random bed,
    tau* ~ 1), with the Darcy-Weisbach or the Manning (Strickler) form of
    tau*: 192 x 96, 100 steps."""
    w = W.antidune2d(nx=192, ny=96, seed=1)
    w["params"].update(bedload=law)
    if fric == "strickler":
        w["params"].update(friction="strickler", K_st=40.0)
    got = run_gpu(w, 100)
    ref = run_orc(w, 100)
    assert_parity(got, ref, 2, ctx=f"{law}/{fric}")
    assert np.max(np.abs(ref["z"] - w["z"])) > 1e-6  # the bed moved


@pytest.mark.parametrize("nx,ny,bc,extra", [
    (97, 45, ("periodic", "periodic", "periodic", "periodic"), dict()),
    (65, 33, ("wall", "wall", "wall", "wall"), dict(friction="darcy", f_dw=0.03)),
    (33, 9, ("inflow_qh", "free", "wall", "free"), dict(q_in=0.9, h_in=1.9, friction="strickler", K_st=40.0)),
    (31, 7, ("inflow_q", "free", "free", "free"), dict(q_in=0.5)),
])
def test_fp32_state_ragged_tiles_and_boundaries(nx, ny, bc, extra):
    """The FP32 2D step (30-column strips marching over runs of rows) on
    grids that leave partial strips and runs at the right and top edges, or
    are narrower than one strip, under every boundary rule: error against the FP64 oracle after 150 steps within the
    FP32 bounds, masses conserved (to FP32 rounding) on the closed and
    periodic grids."""
    w = W.random_smooth(nx, ny, seed=nx + ny, bc=bc, A_g=0.02, **extra)
    got = run_gpu(w, 150, precision="fp32")
    ref = run_orc(w, 150)
    qscale = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])))
    assert rel_err(got["h"], ref["h"]) <= 1e-4
    assert rel_err(got["z"], ref["z"]) <= 1e-4
    assert rel_err(got["hu"], ref["hu"], qscale) <= 1e-3
    assert rel_err(got["hv"], ref["hv"], qscale) <= 1e-3
    if bc[0] in ("periodic", "wall") and bc[2] in ("periodic", "wall"):
        # conserved to FP32 rounding: at a wall the z flux of the mirrored
        # Riemann problem vanishes only up to the float rounding of the solve
        # (~eps_f32 per wall interface and step; FP64: 1e-13, tested above)
        p = w["params"]
        cell = (p["lx"] / nx) * (p["ly"] / ny)
        assert got["diag"]["mass_h"] == pytest.approx(np.sum(w["h"]) * cell, rel=1e-5)
        assert got["diag"]["mass_z"] == pytest.approx(np.sum(w["z"]) * cell, rel=1e-5)


def test_fp32_state_fixed_steps_and_errors():
    """The FP32 2D step with recorded time steps (sve_step_dt) follows the
    FP64 oracle run with the same steps; a step far above the CFL limit
    latches a state error (no trap) and the handle stays usable."""
    w = W.random_smooth(70, 37, seed=3, bc=("inflow_q", "free", "wall", "free"), A_g=0.02, q_in=0.3)
    dts = np.full(120, 0.05)
    got = run_gpu(w, 120, precision="fp32", dts=dts)
    ref = run_orc(w, 120, dts=dts)
    assert np.array_equal(got["dts"], dts)
    qscale = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])))
    assert rel_err(got["h"], ref["h"]) <= 1e-4
    assert rel_err(got["z"], ref["z"]) <= 1e-4
    assert rel_err(got["hu"], ref["hu"], qscale) <= 1e-3
    s = sve.Solver(w["params"], "fp32")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    with pytest.raises(sve.SveError) as e:
        s.step_dt(np.full(4, 60.0))
    assert e.value.code in (sve.SVE_ERR_NEG_DEPTH, sve.SVE_ERR_NAN, sve.SVE_ERR_RIEMANN, sve.SVE_ERR_DT)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(10)
    out = s.get_state()
    s.close()
    assert np.all(np.isfinite(out["h"])) and np.all(out["h"] > 0)


@pytest.mark.parametrize("law", ["nielsen", "camenen"])
def test_shields_laws_fp32_state(law):
    w = W.antidune2d(nx=256, ny=128, seed=4)
    w["params"].update(bedload=law)
    got = run_gpu(w, 200, precision="fp32")
    ref = run_orc(w, 200)
    qscale = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])))
    assert rel_err(got["h"], ref["h"]) <= 1e-4
    assert rel_err(got["z"], ref["z"], scale=max(np.max(np.abs(ref["z"])), 1e-2)) <= 1e-4
    assert rel_err(got["hu"], ref["hu"], qscale) <= 1e-3


@pytest.mark.parametrize("A_g", [1.0, 0.1])
def test_paper_bump2d_reduced_grid(A_g):
    """The 2D bump of Sec. 5.3 (1000 x 1000 m, q0 = 10, 2D Grass m_g = 3,
    inflow upstream, free flow elsewhere) on a 200 x 200 grid, 200 steps."""
    w = W.paper_bump2d(nx=200, ny=200, A_g=A_g)
    got = run_gpu(w, 200)
    ref = run_orc(w, 200)
    assert_parity(got, ref, 2, ctx=f"bump A_g={A_g}")
    assert abs(got["t"] - ref["t"]) <= 1e-10 * ref["t"]


def test_c3_full_grid_first_dt():
    """The full antidune grid (8192 x 4096): the first CFL step equals the
    oracle's CFL step of the initial state, and one step stays finite and
    positive."""
    w = W.antidune2d()
    P = oracle.Params.from_workload(w["params"])
    dt_ref = oracle.get().cfl(P, w["h"], w["hu"], w["hv"], w["z"])
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(1)
    dts = s.dts(1)
    st = s.get_state()
    s.close()
    assert abs(dts[0] - dt_ref) <= 1e-12 * dt_ref
    assert np.all(st["h"] > 0) and np.all(np.isfinite(st["z"]))


def test_fixed_dt_and_y_invariance():
    """Fixed steps (sve_step_dt): 2D on y-invariant data with the 1D run's
    steps reproduces the 1D run in every row (oracle property, GPU path)."""
    w1 = W.dune1d(nx=300, nsteps=400)
    w1["params"]["lx"] = 300.0
    g1 = run_gpu(w1, 400)
    ny = 7
    p2 = dict(w1["params"])
    p2.update(dim=2, ny=ny, ly=7.0, bc=("periodic",) * 4)
    w2 = dict(params=p2, h=np.tile(w1["h"], (ny, 1)), hu=np.tile(w1["hu"], (ny, 1)), hv=np.zeros((ny, 300)),
              z=np.tile(w1["z"], (ny, 1)))
    g2 = run_gpu(w2, 400, dts=g1["dts"])
    for k in ("h", "hu", "z"):
        assert rel_err(g2[k], np.tile(g1[k], (ny, 1))) <= 1e-13
    assert np.all(g2["hv"] == 0)


def test_mass_conservation_gpu():
    """Periodic 2D domain: water and sediment mass sums (FP64 device
    reductions) stay constant."""
    w = W.random_smooth(150, 70, seed=21, bc=("periodic",) * 4, A_g=0.05)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    d0 = s.diag()
    s.step(500)
    d1 = s.diag()
    s.close()
    assert abs(d1["mass_h"] - d0["mass_h"]) <= 1e-13 * d0["mass_h"]
    assert abs(d1["mass_z"] - d0["mass_z"]) <= 1e-13 * d0["mass_z"]


def test_device_pointers_and_stream():
    """State in and out as CUDA tensors on a side stream."""
    import torch

    w = W.dune2d(nx=90, ny=40, seed=2, lx=90.0, ly=40.0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        t = {k: torch.tensor(w[k], dtype=torch.float64, device="cuda") for k in ("h", "hu", "hv", "z")}
        s = sve.Solver(w["params"], "fp64", stream=stream.cuda_stream)
        s.set_state(t["h"], t["hu"], t["hv"], t["z"])
        s.step(50)
        out = {k: torch.empty_like(t[k]) for k in t}
        s.get_state_device(out["h"], out["hu"], out["hv"], out["z"])
    stream.synchronize()
    ref = run_orc(w, 50)
    got = {k: out[k].cpu().numpy() for k in out}
    assert_parity(got, ref, 2, ctx="device pointers")
    s.close()


def test_errors_latched_not_trapped():
    """A state with a non-positive depth is rejected by sve_set_state; the
    handle stays usable afterwards."""
    w = W.dune2d(nx=40, ny=20, seed=1, lx=40.0, ly=20.0)
    s = sve.Solver(w["params"], "fp64")
    bad = w["h"].copy()
    bad[3, 7] = -1.0
    with pytest.raises(sve.SveError) as e:
        s.set_state(bad, w["hu"], w["hv"], w["z"])
    assert e.value.code == sve.SVE_ERR_NEG_DEPTH
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(5)
    s.close()


@pytest.mark.parametrize("case", ["dune2d", "antidune2d"])
def test_fp32_state_error_vs_fp64_oracle(case):
    """FP32 state: relative L-infinity error against the FP64 oracle after
    200 steps stays below 1e-4 (h, z) / 1e-3 (discharges)."""
    if case == "dune2d":
        w = W.dune2d(nx=160, ny=80, seed=4)
    else:
        w = W.antidune2d(nx=256, ny=128, seed=4)
    got = run_gpu(w, 200, precision="fp32")
    ref = run_orc(w, 200)
    qscale = max(np.max(np.abs(ref["hu"])), np.max(np.abs(ref["hv"])))
    assert rel_err(got["h"], ref["h"]) <= 1e-4
    assert rel_err(got["z"], ref["z"], scale=max(np.max(np.abs(ref["z"])), 1e-2)) <= 1e-4
    assert rel_err(got["hu"], ref["hu"], qscale) <= 1e-3
    assert rel_err(got["hv"], ref["hv"], qscale) <= 1e-3
