"""The discrete adjoint (sve_record_forward / sve_adjoint) through the C ABI
against central finite differences of the GPU forward run with the recorded
time steps held fixed, and the torch.autograd.Function built on it."""
from __future__ import annotations

import numpy as np
import pytest

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


def case(bc=("inflow_q", "free", "wall", "free"), friction="strickler"):
    """Smooth random state (no two neighbours equal: the discrete map is
    differentiable there -- at exact ties of the celerity maxima it has
    kinks, where central differences and the one-sided adjoint differ)."""
    w = W.random_smooth(40, 24, seed=7, bc=bc, A_g=5e-3, m_g=3.1, q_in=0.3, friction="strickler", K_st=40.0)
    if friction == "darcy":
        w["params"].update(friction="darcy", f_dw=0.03)
    rng = np.random.default_rng(1)
    target = w["z"] + 0.01 * rng.standard_normal(w["z"].shape)
    return w, target


def forward_fixed(w, p, dts, z0=None, h0=None):
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"] if h0 is None else h0, w["hu"], w["hv"], w["z"] if z0 is None else z0)
    s.step_dt(dts)
    out = s.get_state()
    s.close()
    return out


def loss(out, target):
    return float(np.sum((out["z"] - target) ** 2))


@pytest.mark.parametrize("bc,friction,every", [
    (("inflow_q", "free", "wall", "free"), "strickler", 7),
    (("periodic", "periodic", "periodic", "periodic"), "darcy", 0),
])
def test_adjoint_vs_central_differences(bc, friction, every):
    w, target = case(bc, friction)
    p = w["params"]
    n = 30
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, every)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    # the recorded steps: rerun the CFL forward once to read them
    s2 = sve.Solver(p, "fp64")
    s2.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s2.step(n)
    dts = s2.dts(n)
    s2.close()
    # parameters, with relative steps of 1e-6 (A_g, m_g) and 1e-4 (the weakly
    # coupled friction coefficient: at 1e-6 the loss moves by ~1e-12, where
    # the forward map's rounding -- piecewise constant at the ulp level --
    # puts ~1e-4 relative noise into the difference quotient)
    coef_name = "K_st" if friction == "strickler" else "f_dw"
    for idx, name in enumerate(("A_g", "m_g", coef_name)):
        v = p[name]
        e = (1e-4 if name == coef_name else 1e-6) * abs(v)
        pp, pm = dict(p), dict(p)
        pp[name] = v + e
        pm[name] = v - e
        fd = (loss(forward_fixed(w, pp, dts), target) - loss(forward_fixed(w, pm, dts), target)) / (2 * e)
        assert abs(gp[idx] - fd) <= 1e-5 * max(abs(fd), 1e-12) + 1e-9, (name, gp[idx], fd)
    # initial bed and depth, along smooth random directions
    rng = np.random.default_rng(2)
    X, Y = np.meshgrid(np.linspace(0, 1, p["nx"]), np.linspace(0, 1, p["ny"]))
    for field, key in (("z", "z"), ("h", "h")):
        d = np.sin(2 * np.pi * (rng.uniform(1, 3) * X + rng.uniform(0, 2) * Y) + rng.uniform(0, 6))
        e = 1e-6
        kw_p = {("z0" if key == "z" else "h0"): w[key] + e * d}
        kw_m = {("z0" if key == "z" else "h0"): w[key] - e * d}
        fd = (loss(forward_fixed(w, p, dts, **kw_p), target) - loss(forward_fixed(w, p, dts, **kw_m), target)) / (2 * e)
        ad = float(np.sum(grads[field] * d))
        assert abs(ad - fd) <= 1e-5 * abs(fd) + 1e-9, (field, ad, fd)


def test_autograd_function_matches_adjoint():
    import torch

    from paper_1307_0491_gb300.autograd import bed_evolution

    w, target = case()
    p = w["params"]
    dev = "cuda"
    T = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    z0 = T(w["z"]).requires_grad_(True)
    A = T(p["A_g"]).requires_grad_(True)
    m = T(p["m_g"]).requires_grad_(True)
    K = T(p["K_st"]).requires_grad_(True)
    zT = bed_evolution(z0, A, m, K, p, T(w["h"]), T(w["hu"]), T(w["hv"]), 25, 5)
    L = torch.sum((zT - T(target)) ** 2)
    L.backward()
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(25, 5)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    assert np.allclose(z0.grad.cpu().numpy(), grads["z"], rtol=1e-12, atol=1e-15)
    assert np.allclose([A.grad.item(), m.grad.item(), K.grad.item()], gp, rtol=1e-12)


@pytest.mark.parametrize("bc,friction", [
    (("inflow_q", "free", "wall", "free"), "strickler"),
    (("periodic", "periodic", "periodic", "periodic"), "darcy"),
])
def test_gpu_adjoint_equals_oracle_adjoint(bc, friction):
    """GPU adjoint against the oracle-side adjoint (autograd through the
    PyTorch-CPU restatement of the step), each from its own forward run and
    its own CFL time steps: 1e-10 relative."""
    pytest.importorskip("torch")
    import oracle
    from oracle import adjoint as OA

    w, target = case(bc, friction)
    p = w["params"]
    n = 20
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, 6)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    ref = oracle.get().run(oracle.Params.from_workload(p), n, w["h"], w["hu"], w["hv"], w["z"])
    og = OA.gradients(p, w, ref["dts"], 2.0 * (np.asarray(ref["z"]) - target))
    # relative L-infinity over the gradient with respect to the initial state,
    # and over the parameter gradient (A_g, m_g, friction coefficient)
    scale = max(np.max(np.abs(og["z"])), np.max(np.abs(og["h"])))
    errs = {f: float(np.max(np.abs(grads[f] - og[f])) / scale) for f in ("z", "h")}
    pscale = max(abs(b) for b in og["params"])
    perr = [abs(a - b) / pscale for a, b in zip(gp, og["params"])]
    print("adjoint vs oracle adjoint:", errs, perr)
    assert max(errs.values()) <= 1e-10, errs
    assert max(perr) <= 1e-10, (gp, og["params"])


def test_stepping_after_the_adjoint():
    """After sve_adjoint the handle holds the recorded run's initial state:
    stepping on from there equals stepping from that state afresh."""
    w, target = case()
    p = w["params"]
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(25, 5)
    fin = s.get_state()
    s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.step(15)
    after = s.get_state()
    s.close()
    s2 = sve.Solver(p, "fp64")
    s2.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s2.step(15)
    ref = s2.get_state()
    s2.close()
    for k in ("h", "hu", "hv", "z"):
        assert np.max(np.abs(after[k] - ref[k])) <= 1e-12 * max(np.max(np.abs(ref[k])), 1e-300), k


def test_stored_and_checkpointed_recordings_agree():
    """The automatic recording keeps every step on a grid this small
    (checkpoint interval = nsteps, no recompute); with checkpoints every 5 or
    23 steps the segments are recomputed in fixed-dt mode.  The same kernels
    with the same time steps: final states and gradients equal bit for bit,
    and the handle steps on from U^0 afterwards in each mode."""
    w, target = case()
    p = w["params"]
    n = 23
    out = {}
    for every in (0, 5, 23):
        s = sve.Solver(p, "fp64")
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        s.record_forward(n, every)
        ce = s.checkpoint_every()
        fin = s.get_state()
        grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
        s.step(4)
        after = s.get_state()
        s.close()
        out[every] = (ce, fin, grads, gp, after)
    assert out[0][0] == n and out[5][0] == 5 and out[23][0] == 23
    for every in (5, 23):
        for k in ("h", "hu", "hv", "z"):
            assert np.array_equal(out[every][1][k], out[0][1][k]), (every, k)
            assert np.array_equal(out[every][2][k], out[0][2][k]), (every, k)
            assert np.array_equal(out[every][4][k], out[0][4][k]), (every, k)
        assert list(out[every][3]) == list(out[0][3])


def test_partly_kept_recording_agrees():
    """An automatic recording whose memory budget holds the last two
    checkpoint segments' forward data (23 steps: segments of 5, 5, 5, 5, 3
    steps, the last 8 kept) recomputes only the first three in the reverse
    sweep; with a zero budget it keeps nothing.  Final states, gradients and
    the state stepped on from U^0 afterwards equal those of the recording
    that keeps every step, bit for bit."""
    w, target = case()
    p = w["params"]
    nx, ny = p["nx"], p["ny"]
    n, every = 23, 5
    npad = (nx + 2) * (ny + 2)
    nf = (nx + 1) * ny + nx * (ny + 1)
    per_step = 8 * (4 * npad + 4 * nx * ny + nf) + nf
    ncp = -(-n // every)
    out = {}
    for name, budget in (("all", -1), ("two", per_step * (every + 8) + 8 * 4 * npad * ncp + 64), ("none", 0)):
        s = sve.Solver(p, "fp64")
        s.set_adjoint_budget(budget)
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        s.record_forward(n, 0)
        kept, ce = s.adjoint_kept_steps(), s.checkpoint_every()
        fin = s.get_state()
        grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
        s.step(4)
        after = s.get_state()
        s.close()
        out[name] = (kept, ce, fin, grads, gp, after)
    assert out["all"][:2] == (n, n)
    assert out["two"][:2] == (8, every)
    assert out["none"][:2] == (0, every)
    for name in ("two", "none"):
        for k in ("h", "hu", "hv", "z"):
            for i in (2, 3, 5):
                assert np.array_equal(out[name][i][k], out["all"][i][k]), (name, i, k)
        assert list(out[name][4]) == list(out["all"][4])


def shields_case(law, friction, bc):
    """A Shields-parameter law on a supercritical channel with a rippled bed,
    a small random transverse flow and a depth perturbed by 0.1 mm (tau*
    around 1: above the threshold).  The antidune config's uniform depth
    would make the celerity maxima of Eq. (ab) tie at every interface, where
    the discrete map has kinks in h and the adjoint and the oracle's autograd
    take different one-sided derivatives."""
    w = W.antidune2d(nx=40, ny=24, seed=51)
    w["params"].update(bedload=law, friction=friction, f_dw=0.02, K_st=40.0, bc=bc)
    rng = np.random.default_rng(52)
    w["hv"] = 0.02 * rng.standard_normal(np.shape(w["h"]))
    w["h"] = w["h"] + 1e-4 * rng.standard_normal(np.shape(w["h"]))
    target = w["z"] + 0.002 * rng.standard_normal(np.shape(w["z"]))
    return w, target


@pytest.mark.parametrize("law,friction,bc", [
    ("mpm", "darcy", ("inflow_qh", "free", "wall", "free")),
    ("mpm", "strickler", ("periodic",) * 4),
    ("flvb", "darcy", ("periodic",) * 4),
    ("nielsen", "strickler", ("inflow_qh", "free", "free", "free")),
    ("ribberink", "darcy", ("periodic",) * 4),
    ("camenen", "strickler", ("periodic",) * 4),
])
def test_shields_adjoint_equals_oracle_adjoint(law, friction, bc):
    """The Shields-parameter laws in the adjoint (their q*, dq*/dtau* and
    d2q*/dtau*2 in the reverse sweep; tau* through the friction
    coefficient): GPU against the oracle-side adjoint, 1e-10 relative."""
    import oracle
    from oracle import adjoint as OA

    w, target = shields_case(law, friction, bc)
    p = w["params"]
    n = 15
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, 0)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    ref = oracle.get().run(oracle.Params.from_workload(p), n, w["h"], w["hu"], w["hv"], w["z"])
    og = OA.gradients(p, w, ref["dts"], 2.0 * (np.asarray(ref["z"]) - target))
    scale = max(np.max(np.abs(og["z"])), np.max(np.abs(og["h"])))
    errs = {f: float(np.max(np.abs(grads[f] - og[f])) / scale) for f in ("z", "h")}
    assert max(errs.values()) <= 1e-10, errs
    assert gp[0] == 0.0 and gp[1] == 0.0
    assert abs(gp[2] - og["params"][2]) <= 1e-10 * abs(og["params"][2]), (gp, og["params"])


def test_shields_adjoint_vs_central_differences():
    """MPM with Strickler friction (tau* with h^(-1/3)): the friction
    coefficient's gradient (through the friction and through tau*) and a bed
    direction against central differences of the GPU forward run."""
    w, target = shields_case("mpm", "strickler", ("periodic",) * 4)
    p = w["params"]
    n = 15
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, 4)
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    s2 = sve.Solver(p, "fp64")
    s2.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s2.step(n)
    dts = s2.dts(n)
    s2.close()
    v = p["K_st"]
    e = 1e-5 * v
    pp, pm = dict(p), dict(p)
    pp["K_st"], pm["K_st"] = v + e, v - e
    fd = (loss(forward_fixed(w, pp, dts), target) - loss(forward_fixed(w, pm, dts), target)) / (2 * e)
    assert abs(gp[2] - fd) <= 1e-6 * abs(fd), (gp[2], fd)
    rng = np.random.default_rng(53)
    d = rng.uniform(-1, 1, np.shape(w["z"]))
    # a small step: with the small transverse flow the contact speed of some
    # y-interfaces is near zero, where the fan's wave count (and the map's
    # slope) changes; the difference quotient's error from such crossings
    # shrinks with the step (as in the oracle-side checks)
    e = 1e-8
    fd = (loss(forward_fixed(w, p, dts, z0=w["z"] + e * d), target) -
          loss(forward_fixed(w, p, dts, z0=w["z"] - e * d), target)) / (2 * e)
    ad = float(np.sum(grads["z"] * d))
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


@pytest.mark.parametrize("every", [6, 0])
def test_adjoint_through_halvings_and_doublings(every):
    """Colliding supercritical streams (1D, 20 steps from the meeting): the
    forward solves halve Newton steps and double the celerity a; the value
    pass starts from the roots (and doublings) the recording or the
    segment's recompute kept.  GPU adjoint against the oracle-side adjoint
    (which solves and retries on its own), with checkpoints every 6 steps
    and with every step kept."""
    pytest.importorskip("torch")
    import oracle
    from oracle import adjoint as OA

    w = W.colliding_streams(60, m_g=3.1)
    p = w["params"]
    rng = np.random.default_rng(3)
    # depths and discharges perturbed by 0.1 % and m_g off 3: no ties of the
    # celerity bounds between neighbours (at m_g = 3 the bound g h^2 dQ/du of
    # a uniform discharge does not depend on h; the map has kinks at ties,
    # where the adjoint and autograd take different one-sided derivatives)
    w["h"] = w["h"] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, w["h"].shape))
    w["hu"] = w["hu"] * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, w["hu"].shape))
    target = w["z"] + 0.001 * rng.standard_normal(w["z"].shape)
    n = 20
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.record_forward(n, every)
    sg = s.safeguards()
    fin = s.get_state()
    grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - target))
    s.close()
    assert sg["halvings"] > 0 and sg["retries"] > 0, sg
    ref = oracle.get().run(oracle.Params.from_workload(p), n, w["h"], w["hu"], w["hv"], w["z"])
    og = OA.gradients(p, w, ref["dts"], 2.0 * (np.asarray(ref["z"]) - target))
    scale = max(np.max(np.abs(og["z"])), np.max(np.abs(og["h"])))
    errs = {f: float(np.max(np.abs(grads[f] - og[f])) / scale) for f in ("z", "h")}
    pscale = max(abs(b) for b in og["params"][:2])
    perr = [abs(a - b) / pscale for a, b in zip(gp[:2], og["params"][:2])]
    print("adjoint vs oracle adjoint (colliding streams):", errs, perr)
    assert max(errs.values()) <= 1e-9, errs
    assert max(perr) <= 1e-9, (gp, og["params"])
