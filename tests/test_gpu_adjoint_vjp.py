"""The reverse-mode transposed-Jacobian product of one interface's
fluctuations (interface_vjp, used by the adjoint) against the forward-mode
dual-number Jacobian through the step's own templates (jac_pass), on random
interfaces that reach every fan state that occurs (1..4 waves of negative
speed), the bed-step branch of the celerities and both signs of the
b-waves; and on strong compressions, where the solve halves Newton steps
and doubles the celerity a (the doubling scales a's cotangent)."""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _inputs(n=6000, seed=5):
    rng = np.random.default_rng(seed)
    rows = []
    for k in range(n):
        HL, HR = rng.uniform(0.2, 3.0, 2)
        cL, cR = np.sqrt(9.81 * HL), np.sqrt(9.81 * HR)
        kind = k % 4
        if kind == 0:  # subcritical
            uL, uR = rng.uniform(-0.6, 0.6, 2) * (cL, cR)
        elif kind == 1:  # supercritical to the right / to the left, similar depths
            HR = HL * rng.uniform(0.95, 1.05)
            cR = np.sqrt(9.81 * HR)
            s = 1 if rng.random() < 0.5 else -1
            uL, uR = s * rng.uniform(1.6, 3.0, 2) * (cL, cR)
        elif kind == 2:  # shocks and rarefactions
            uL, uR = rng.uniform(-2.0, 2.0, 2) * (cL, cR)
        else:  # near-critical over a bed step
            uL, uR = rng.uniform(0.8, 1.2, 2) * (cL, cR)
        vL, vR = rng.uniform(-0.5, 0.5, 2)
        ZL = rng.uniform(0.0, 0.3)
        ZR = ZL + (rng.uniform(-0.4, 0.4) * min(HL, HR) if kind == 3 else rng.uniform(-0.05, 0.05))
        A = 10.0 ** rng.uniform(-3, -0.5)
        m = rng.choice([1.5, 2.0, 2.5, 3.0, 3.3, 4.0])
        bars = rng.standard_normal(8)
        rows.append([HL, HL * uL, HL * vL, ZL, HR, HR * uR, HR * vR, ZR, A, m, *bars])
    return np.array(rows)


def _hard_inputs(n=2000, seed=7):
    """Colliding states (u_L > 0 > u_R, depths 1 mm .. 10 m): hydraulic-jump
    compressions."""
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(n):
        HL, HR = 10 ** rng.uniform(-3, 1, 2)
        uL, uR = rng.uniform(0.5, 8), rng.uniform(-8, -0.5)
        vL, vR = rng.uniform(-0.5, 0.5, 2)
        ZL, ZR = rng.uniform(-1, 1, 2) * rng.choice([0.0, 0.01, 0.1])
        A = 10.0 ** rng.uniform(-4, 0)
        m = rng.choice([1.0, 2.0, 3.0, 4.0])
        rows.append([HL, HL * uL, HL * vL, ZL, HR, HR * uR, HR * vR, ZR, A, m, *rng.standard_normal(8)])
    return np.array(rows)


def _run_driver(x):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "vjp_driver")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                        os.path.join(HERE, "gpu_adjoint_driver.cu")], check=True)
        r = subprocess.run([exe], input="\n".join(" ".join(repr(float(v)) for v in row) for row in x),
                           capture_output=True, text=True, check=True)
    out = np.array([[float(t) for t in line.split()] for line in r.stdout.splitlines()])
    assert out.shape == (x.shape[0], 27)
    return out


def test_reverse_mode_matches_dual_numbers():
    x = _inputs()
    out = _run_driver(x)
    ok = out[:, 0] == 1.0
    assert ok.mean() > 0.9
    fwd, rev = out[ok, 1:11], out[ok, 11:21]
    # every fan state that can occur and the bed-step branch are covered: the
    # outer waves always straddle x/t = 0 (a >= kappa_a b0 >= kappa_a |H u_n|,
    # so a tau > |u_n|), so 1..4 waves have negative speed, never 0 or 5
    states = set(out[ok, 21].astype(int).tolist())
    assert states == {1, 2, 3, 4}, states
    assert np.any(out[ok, 22] == 1.0)
    scale = np.maximum(np.max(np.abs(fwd), axis=1, keepdims=True), 1e-300)
    rel = np.max(np.abs(rev - fwd) / scale, axis=1)
    assert np.max(rel) <= 1e-10, (np.max(rel), np.argmax(rel))
    assert np.median(rel) <= 1e-13
    # each output on its own scale (the A_g and m_g components are small
    # next to the state components of the same interface)
    for k in range(10):
        ck = np.abs(rev[:, k] - fwd[:, k]) / np.maximum(np.abs(fwd[:, k]), 1e-12 * np.max(np.abs(fwd[:, k])))
        assert np.median(ck) <= 1e-12, (k, np.median(ck))
        assert np.quantile(ck, 0.99) <= 1e-9, (k, np.quantile(ck, 0.99))


def test_reverse_mode_on_strong_compressions():
    """Hydraulic-jump compressions: the value pass repeats the step's halved
    Newton steps and doublings of a, and the reverse mode still equals the
    forward-mode dual numbers through the same solve (relative to each
    interface's largest output; these solves are ill conditioned -- tau_k
    spans up to four decades -- so the bound is looser than on smooth
    states)."""
    x = _hard_inputs()
    out = _run_driver(x)
    ok = out[:, 0] == 1.0
    assert ok.mean() > 0.99
    assert np.sum(out[ok, 24] > 0) >= 50 and np.sum(out[ok, 25] > 0) >= 50, (
        np.sum(out[ok, 24] > 0), np.sum(out[ok, 25] > 0))
    fwd, rev = out[ok, 1:11], out[ok, 11:21]
    scale = np.maximum(np.max(np.abs(fwd), axis=1, keepdims=True), 1e-300)
    rel = np.max(np.abs(rev - fwd) / scale, axis=1)
    retried = out[ok, 24] > 0
    spread = out[ok, 26]
    q = {f"q{int(100 * f)}": float(np.quantile(rel, f)) for f in (0.5, 0.9, 0.99)}
    info = dict(**q, max=float(rel.max()), spread_at_max=float(spread[np.argmax(rel)]),
                spread_q99=float(np.quantile(spread, 0.99)))
    # a wrong cotangent of a through its doublings would be O(1) in most
    # retried rows; rounding in these solves grows with the spread of tau
    assert np.median(rel[retried]) <= 1e-11, info
    assert np.median(rel) <= 1e-11 and q["q90"] <= 1e-7, info
    assert q["q99"] <= 1e-4 and info["max"] <= 1e-2, info
