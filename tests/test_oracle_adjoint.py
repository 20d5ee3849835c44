"""Pins of the oracle-side adjoint (oracle/adjoint.py, a PyTorch-CPU FP64
restatement of the step differentiated by autograd): its forward equals the
C oracle's, and its gradients equal central differences of the C oracle's
forward with the time steps held fixed."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import workloads as W

torch = pytest.importorskip("torch")
from oracle import adjoint as OA  # noqa: E402


def case(dim=2, bc=("inflow_q", "free", "wall", "free"), friction="strickler", law="grass"):
    if law != "grass":
        # a Shields-parameter law on a supercritical channel with a rippled
        # bed (tau* around 1, above the threshold everywhere)
        w = W.antidune2d(nx=12, ny=8, seed=43)
        w["params"].update(bedload=law, friction=friction, f_dw=0.02, K_st=40.0, bc=bc if bc[0] != "inflow_q"
                           else ("inflow_qh", "free", "wall", "free"))
        rng = np.random.default_rng(44)
        w["hv"] = 0.02 * rng.standard_normal(np.shape(w["h"]))
        return w
    if dim == 2:
        w = W.random_smooth(12, 8, seed=41, bc=bc, A_g=5e-3, m_g=3.1, q_in=0.3, friction=friction, K_st=40.0,
                            f_dw=0.03)
    else:
        w = W.random_smooth(16, 1, seed=42, dim=1, bc=("periodic",) * 4, A_g=5e-3, m_g=2.4, friction=friction,
                            K_st=35.0, f_dw=0.03)
    return w


def c_oracle(w, dts, **over):
    p = dict(w["params"])
    p.update({k: v for k, v in over.items() if k in p})
    st = {k: (over.get(k + "0", w[k])) for k in ("h", "hu", "hv", "z")}
    return oracle.get().run(oracle.Params.from_workload(p), len(dts), st["h"], st["hu"], st["hv"], st["z"], dts=dts)


CASES = [
    (2, ("inflow_q", "free", "wall", "free"), "strickler", "grass"),
    (2, ("periodic",) * 4, "darcy", "grass"),
    (1, ("periodic",) * 4, "strickler", "grass"),
    (2, ("inflow_q", "free", "wall", "free"), "darcy", "mpm"),
    (2, ("periodic",) * 4, "strickler", "mpm"),
    (2, ("periodic",) * 4, "darcy", "nielsen"),
    (2, ("periodic",) * 4, "strickler", "camenen"),
]


@pytest.mark.parametrize("dim,bc,friction,law", CASES)
def test_torch_forward_equals_c_oracle(dim, bc, friction, law):
    w = case(dim, bc, friction, law)
    p = w["params"]
    dts = oracle.get().run(oracle.Params.from_workload(p), 20, w["h"], w["hu"], w["hv"], w["z"])["dts"]
    ref = c_oracle(w, dts)
    T = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64).reshape(p["ny"] if dim == 2 else 1, p["nx"])
    st = dict(h=T(w["h"]), hu=T(w["hu"]), hv=T(w["hv"]) if dim == 2 else torch.zeros(1, p["nx"], dtype=torch.float64),
              z=T(w["z"]))
    coef = p["K_st"] if friction == "strickler" else p["f_dw"]
    h, hu, hv, z = OA.run(p, st, dts, torch.tensor(p["A_g"], dtype=torch.float64),
                          torch.tensor(p["m_g"], dtype=torch.float64), torch.tensor(coef, dtype=torch.float64))
    for got, key in ((h, "h"), (hu, "hu"), (z, "z")):
        ref_a = np.asarray(ref[key]).reshape(got.shape)
        assert np.max(np.abs(got.numpy() - ref_a)) <= 1e-12 * max(np.max(np.abs(ref_a)), 1e-3), key


@pytest.mark.parametrize("dim,bc,friction,law", CASES)
def test_torch_adjoint_equals_central_differences(dim, bc, friction, law):
    w = case(dim, bc, friction, law)
    p = w["params"]
    n = 15
    dts = oracle.get().run(oracle.Params.from_workload(p), n, w["h"], w["hu"], w["hv"], w["z"])["dts"]
    rng = np.random.default_rng(3)
    target = np.asarray(w["z"]) + 0.01 * rng.standard_normal(np.shape(w["z"]))
    zT = np.asarray(c_oracle(w, dts)["z"])
    g = OA.gradients(p, w, dts, 2.0 * (zT - target))

    def loss(**over):
        return float(np.sum((np.asarray(c_oracle(w, dts, **over)["z"]) - target) ** 2))

    # central differences with relative steps of 1e-5 (A_g, m_g) and 1e-4 (the
    # weakly coupled friction coefficient): larger steps cross kinks of the
    # discrete map (a celerity maximum switching sides), smaller ones are
    # dominated by its rounding noise (measured agreement ~1e-9 .. 1e-7)
    coef_name = "K_st" if friction == "strickler" else "f_dw"
    for idx, name in enumerate(("A_g", "m_g", coef_name)):
        if law != "grass" and name in ("A_g", "m_g"):
            assert g["params"][idx] == 0.0  # the Grass parameters do not enter
            continue
        v = p[name]
        e = (1e-4 if name == coef_name else 1e-5) * abs(v)
        fd = (loss(**{name: v + e}) - loss(**{name: v - e})) / (2 * e)
        assert abs(g["params"][idx] - fd) <= 1e-6 * abs(fd) + 1e-10, (name, g["params"][idx], fd)
    for field in ("z", "h"):
        d = rng.uniform(-1, 1, np.shape(w[field]))
        # the Shields laws' map bends faster in h (the celerity bounds move
        # with tau*): a smaller step there (measured: the difference quotient
        # approaches the adjoint as 4e-4, 2e-6, 6e-8 at 1e-5, 1e-6, 1e-7)
        e = 1e-7 if (law != "grass" and field == "h") else 1e-6
        fd = (loss(**{field + "0": np.asarray(w[field]) + e * d}) -
              loss(**{field + "0": np.asarray(w[field]) - e * d})) / (2 * e)
        ad = float(np.sum(g[field] * d))
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-10, (field, ad, fd)
