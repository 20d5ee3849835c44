"""Oracle-side discrete adjoint: the step of ``sve_oracle.c`` restated with
plain PyTorch CPU operations in FP64, vectorised over the interfaces, and
differentiated by torch.autograd.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).  It follows the
same procedure and readings as the C oracle (Sec. 3: equilibrium projection,
one relaxation Riemann solve per interface, Godunov average; friction, CFL,
ghosts as readings R1--R8 there), with the Grass law written through
exp/log so that A_g and m_g carry derivatives, and the Shields-parameter
laws (q*(tau*) of Sec. 2, tau* through the friction coefficient, which then
carries a derivative through the closure as well as through the friction).  The Newton
iteration runs without gradients to convergence; one final Newton update
with the derivative F'(p) held constant makes the root's derivative the one
of the implicit function theorem, dp = -F_theta / F_p.

Pins (``tests/test_oracle_adjoint.py``): its forward equals the C oracle's
forward; its gradients equal central differences of the C oracle's forward
with the time steps held fixed.
"""
from __future__ import annotations

import torch

_BC = {"periodic": 0, "free": 1, "inflow_q": 2, "inflow_qh": 3, "wall": 4}


def _ghosts(p: dict, H, Hu, Hv, Z):
    """Padded (ny + 2, nx + 2) fields with the ghost rules (reading R7);
    corners are filled with the interior neighbour (never used)."""
    bc = p["bc"]
    dim = p["dim"]

    def rule(s, line):
        h, qu, qv, z = line
        t = bc[s]
        normal_is_u = s < 2
        inward = 1.0 if s in (0, 2) else -1.0
        qn, qt = (qu, qv) if normal_is_u else (qv, qu)
        if t == "inflow_q":
            qn = torch.full_like(qn, inward * p["q_in"])
            qt = torch.zeros_like(qt)
        elif t == "inflow_qh":
            h = torch.full_like(h, p["h_in"])
            qn = torch.full_like(qn, inward * p["q_in"])
            qt = torch.zeros_like(qt)
        elif t == "wall":
            qn = -qn
        qu, qv = (qn, qt) if normal_is_u else (qt, qn)
        return [h, qu, qv, z]

    F = [H, Hu, Hv, Z]
    # x ghosts
    wsrc = [f[:, -1:] if bc[0] == "periodic" else f[:, :1] for f in F]
    esrc = [f[:, :1] if bc[1] == "periodic" else f[:, -1:] for f in F]
    W = rule(0, wsrc)
    E = rule(1, esrc)
    X = [torch.cat([w, f, e], dim=1) for w, f, e in zip(W, F, E)]
    if dim == 2:
        ssrc = [f[-1:, :] if bc[2] == "periodic" else f[:1, :] for f in X]
        nsrc = [f[:1, :] if bc[3] == "periodic" else f[-1:, :] for f in X]
        S = rule(2, ssrc)
        N = rule(3, nsrc)
        X = [torch.cat([s_, f, n_], dim=0) for s_, f, n_ in zip(S, X, N)]
    else:
        X = [torch.cat([f, f, f], dim=0) for f in X]  # rows -1 and 1 unused in 1D
    return X


def _qstar(law: str, ts, tcr: float):
    """q*(tau*) and dq*/dtau* of the Shields-parameter laws of Sec. 2 (as
    orc_qstar), zero below the threshold; the unused branch is evaluated at
    a safe point so that its derivative stays finite."""
    one = torch.ones_like(ts)
    if law == "camenen":
        on = ts > 0
        t = torch.where(on, ts, one)
        e = torch.exp(-4.5 * tcr / t)
        q = 12.0 * t * torch.sqrt(t) * e
        dq = 12.0 * e * (1.5 * torch.sqrt(t) + 4.5 * tcr / torch.sqrt(t))
    else:
        x = ts - tcr
        on = x > 0
        xs = torch.where(on, x, one)
        t = torch.where(on, ts, one)
        if law in ("mpm", "flvb"):
            c = 8.0 if law == "mpm" else 5.7
            q = c * xs * torch.sqrt(xs)
            dq = c * 1.5 * torch.sqrt(xs)
        elif law == "nielsen":
            q = 12.0 * torch.sqrt(t) * xs
            dq = 12.0 * (xs / (2.0 * torch.sqrt(t)) + torch.sqrt(t))
        elif law == "ribberink":
            q = 11.0 * torch.pow(xs, 1.65)
            dq = 11.0 * 1.65 * torch.pow(xs, 0.65)
        else:
            raise ValueError(law)
    zero = torch.zeros_like(ts)
    return torch.where(on, q, zero), torch.where(on, dq, zero)


def _project(p, H, Hn, Ht, Z, A, m, K):
    g = p["g"]
    tau = 1.0 / H
    un = Hn * tau
    ut = Ht * tau
    Pi = 0.5 * g * H * H
    speed2 = un * un + ut * ut
    zero = speed2 == 0
    sp = torch.sqrt(torch.where(zero, torch.ones_like(speed2), speed2))
    law = p.get("bedload", "grass")
    if law == "grass":
        lsp = torch.log(sp)
        pm1 = torch.exp((m - 1.0) * lsp)
        pm3 = torch.exp((m - 3.0) * lsp)
        Q = torch.where(zero, torch.zeros_like(speed2), A * un * pm1)
        dQ = torch.where(zero, torch.zeros_like(speed2), A * (pm1 + (m - 1.0) * un * un * pm3))
    else:
        # tau* = alpha |U|^2 for the friction law in use (K: its coefficient)
        sm1 = p["s"] - 1.0
        if p["friction"] == "darcy":
            alpha = K / (8.0 * g * sm1 * p["d_s"])
        else:
            n = 1.0 / K
            alpha = (n * n) / (sm1 * p["d_s"] * torch.pow(H, 1.0 / 3.0))
        q, dq = _qstar(law, alpha * speed2, p["tau_cr"])
        on = (~zero) & ((q != 0) | (dq != 0))
        Cs = (sm1 * g * p["d_s"] ** 3) ** 0.5
        Q = torch.where(on, Cs * q * (un / sp), torch.zeros_like(speed2))
        dQ = torch.where(on, Cs * (2.0 * dq * alpha * (un * un) / sp + q * (ut * ut) / (speed2 * sp)),
                         torch.zeros_like(speed2))
    ca = H * torch.sqrt(g * H)
    cb = torch.sqrt(Hn * Hn + g * H * H * dQ)
    return dict(H=H, Hn=Hn, Ht=Ht, Z=Z, tau=tau, un=un, ut=ut, Pi=Pi, Om=Q, ca=ca, cb=cb)


def _eval(p_, c, L, R):
    """Intermediate states and F at p (relations of the five waves)."""
    a, b, K, D = c["a"], c["b"], c["K"], c["D"]
    sigma = (c["du"] + a * (L["tau"] + R["tau"]) - (a - b) * p_) / b
    tau2 = 0.5 * (sigma - D)
    tau3 = 0.5 * (sigma + D)
    N = c["dZ"] + K * D * sigma
    m = -N / (K * p_)
    tau1 = 0.5 * (p_ + m)
    tau4 = 0.5 * (p_ - m)
    u1 = L["un"] + a * (tau1 - L["tau"])
    u4 = R["un"] - a * (tau4 - R["tau"])
    lam2 = u1 - b * tau1
    lam4 = u4 + b * tau4
    Zs = L["Z"] + K * (tau2 * tau2 - tau1 * tau1)
    F = (L["Om"] - R["Om"]) + lam2 * (Zs - L["Z"]) - lam4 * (Zs - R["Z"])
    return dict(tau1=tau1, tau2=tau2, tau3=tau3, tau4=tau4, u1=u1, u4=u4, lam2=lam2, lam4=lam4, Zs=Zs, F=F)


def _dF(p_, c, L, R):
    """F'(p) by a forward derivative through _eval (p as the only variable)."""
    with torch.enable_grad():
        q = p_.detach().clone().requires_grad_(True)
        e = _eval(q, {k: v.detach() for k, v in c.items()}, {k: v.detach() for k, v in L.items()},
                  {k: v.detach() for k, v in R.items()})
        (g,) = torch.autograd.grad(e["F"].sum(), q)
    return g


def riemann(p, L, R, tol=1e-9, maxit=30):
    """Fluctuations (A-, A+) of (H, Hn, Ht, Z) at every interface."""
    g = p["g"]
    a0 = torch.maximum(L["ca"], R["ca"])
    b0 = torch.maximum(L["cb"], R["cb"])
    a = p["kappa_a"] * torch.maximum(a0, b0)
    b = torch.maximum(b0, p["beta_min"] * a0)
    Hmax = torch.maximum(L["H"], R["H"])
    need = b * b + 2.0 * g * p["gamma_z"] * torch.abs(R["Z"] - L["Z"]) * Hmax * Hmax
    a = torch.where(a * a < need, torch.sqrt(need), a)
    same = (L["H"] == R["H"]) & (L["Hn"] == R["Hn"]) & (L["Ht"] == R["Ht"]) & (L["Z"] == R["Z"])
    Ld = {k: v.detach() for k, v in L.items()}
    Rd = {k: v.detach() for k, v in R.items()}
    # Newton to convergence without gradients (reading R2); where the
    # celerities admit no root with positive tau_k, a is doubled and the
    # iteration restarted, at most three times (reading R12)
    for attempt in range(4):
        K = (a * a - b * b) / (2.0 * g)
        D = (R["tau"] - L["tau"]) + (R["Pi"] - L["Pi"]) / (a * a)
        c = dict(a=a, b=b, K=K, D=D, du=R["un"] - L["un"], dZ=R["Z"] - L["Z"])
        p0 = L["tau"] + R["tau"] + c["du"] / a
        with torch.no_grad():
            cd = {k: v.detach() for k, v in c.items()}
            pp = p0.detach().clone()
            done = torch.zeros_like(pp, dtype=torch.bool)
            for _ in range(maxit):
                e = _eval(pp, cd, Ld, Rd)
                step = -e["F"] / _dF(pp, cd, Ld, Rd)
                step = torch.where(done, torch.zeros_like(step), step)
                halved = torch.zeros_like(done)
                for _h in range(61):
                    t = _eval(pp + step, cd, Ld, Rd)
                    ok = (t["tau1"] > 0) & (t["tau2"] > 0) & (t["tau3"] > 0) & (t["tau4"] > 0)
                    if bool(ok.all()):
                        break
                    step = torch.where(ok, step, 0.5 * step)
                    halved = halved | ~ok
                pp = pp + step
                # only a full Newton step measures the distance to the root
                done = done | (~halved & (step.abs() <= tol * pp))
                if bool(done.all()):
                    break
            t = _eval(pp, cd, Ld, Rd)
            good = same | (done & (t["tau1"] > 0) & (t["tau2"] > 0) & (t["tau3"] > 0) & (t["tau4"] > 0))
            if bool(good.all()) or attempt == 3:
                break
        a = torch.where(good, a, 2.0 * a)
    with torch.no_grad():
        Fp = _dF(pp, cd, Ld, Rd)
    # one Newton update with F' held constant: value ~ the root, derivative
    # of the implicit function theorem
    e0 = _eval(pp, c, L, R)
    pr = pp - e0["F"] / Fp
    e = _eval(pr, c, L, R)
    # fluctuations sum_{lam<0} lam [U], sum_{lam>0} lam [U] over the 5 waves
    us = e["u1"] + b * (e["tau2"] - e["tau1"])
    lam = [L["un"] - a * L["tau"], e["lam2"], us, e["lam4"], R["un"] + a * R["tau"]]
    taus = [e["tau1"], e["tau2"], e["tau3"], e["tau4"]]
    us_ = [e["u1"], us, us, e["u4"]]
    vs = [L["ut"], L["ut"], R["ut"], R["ut"]]
    zs = [L["Z"], e["Zs"], e["Zs"], R["Z"]]
    U = [[L["H"], L["Hn"], L["Ht"], L["Z"]]]
    for k in range(4):
        Hk = 1.0 / taus[k]
        U.append([Hk, Hk * us_[k], Hk * vs[k], zs[k]])
    U.append([R["H"], R["Hn"], R["Ht"], R["Z"]])
    Am = [torch.zeros_like(a) for _ in range(4)]
    Ap = [torch.zeros_like(a) for _ in range(4)]
    for k in range(5):
        lk = lam[k]
        for cc in range(4):
            jump = U[k + 1][cc] - U[k][cc]
            Am[cc] = Am[cc] + torch.where(lk < 0, lk * jump, torch.zeros_like(jump))
            Ap[cc] = Ap[cc] + torch.where(lk > 0, lk * jump, torch.zeros_like(jump))
    # bitwise-identical neighbours: zero fluctuations (reading R3), keeping
    # the derivative of the general formula
    same = (L["H"] == R["H"]) & (L["Hn"] == R["Hn"]) & (L["Ht"] == R["Ht"]) & (L["Z"] == R["Z"])
    Am = [x - torch.where(same, x.detach(), torch.zeros_like(x)) for x in Am]
    Ap = [x - torch.where(same, x.detach(), torch.zeros_like(x)) for x in Ap]
    return Am, Ap


def step(p: dict, h, hu, hv, z, dt: float, A, m, K):
    """One step of size dt; h, hu, hv, z: (ny, nx) tensors (1D: (1, nx));
    A, m, K: scalar tensors (K = the friction coefficient)."""
    dim = p["dim"]
    nx, ny = p["nx"], p["ny"] if dim == 2 else 1
    dx = p["lx"] / nx
    dy = p["ly"] / ny if dim == 2 else 1.0
    H, Hu, Hv, Z = _ghosts(p, h, hu, hv, z)
    # x-interfaces: rows 1..ny, columns (i-1, i) for i = 0..nx
    r = slice(1, ny + 1)
    L = _project(p, H[r, :-1], Hu[r, :-1], Hv[r, :-1], Z[r, :-1], A, m, K)
    R = _project(p, H[r, 1:], Hu[r, 1:], Hv[r, 1:], Z[r, 1:], A, m, K)
    Amx, Apx = riemann(p, L, R)
    acc = [(Apx[c][:, :nx] + Amx[c][:, 1:]) / dx for c in range(4)]
    if dim == 2:
        cs = slice(1, nx + 1)
        L = _project(p, H[:-1, cs], Hv[:-1, cs], Hu[:-1, cs], Z[:-1, cs], A, m, K)
        R = _project(p, H[1:, cs], Hv[1:, cs], Hu[1:, cs], Z[1:, cs], A, m, K)
        Amy, Apy = riemann(p, L, R)
        ay = [(Apy[c][:ny, :] + Amy[c][1:, :]) / dy for c in range(4)]
        acc = [acc[0] + ay[0], acc[1] + ay[2], acc[2] + ay[1], acc[3] + ay[3]]
    Hn = h - dt * acc[0]
    q1 = hu - dt * acc[1]
    q2 = hv - dt * acc[2] if dim == 2 else torch.zeros_like(hu)
    Zn = z - dt * acc[3]
    if p["friction"] != "none":
        qn = torch.sqrt(q1 * q1 + q2 * q2)
        if p["friction"] == "darcy":
            C = K / (8.0 * Hn * Hn)
        else:
            C = p["g"] / (K * K * Hn * Hn * torch.pow(Hn, 1.0 / 3.0))
        den = 1.0 + dt * C * qn
        q1 = q1 / den
        q2 = q2 / den
    return Hn, q1, (q2 if dim == 2 else hv), Zn


def run(p: dict, state: dict, dts, A, m, K):
    """Steps with the given time steps; returns the final (h, hu, hv, z)."""
    h, hu, hv, z = state["h"], state["hu"], state["hv"], state["z"]
    for dt in dts:
        h, hu, hv, z = step(p, h, hu, hv, z, float(dt), A, m, K)
    return h, hu, hv, z


def gradients(p: dict, w: dict, dts, lam_z):
    """dL/dz0, dL/dh0 and dL/d(A_g, m_g, K) for L = sum(lam_z * z_T) (the
    cotangent of the final bed), with the time steps held fixed."""
    T = lambda x: torch.tensor(x, dtype=torch.float64)
    shape = (p["ny"], p["nx"]) if p["dim"] == 2 else (1, p["nx"])
    z0 = T(w["z"]).reshape(shape).requires_grad_(True)
    h0 = T(w["h"]).reshape(shape).requires_grad_(True)
    st = dict(h=h0, hu=T(w["hu"]).reshape(shape), hv=(T(w["hv"]).reshape(shape) if p["dim"] == 2
                                                      else torch.zeros(shape, dtype=torch.float64)), z=z0)
    A = T(p["A_g"]).requires_grad_(True)
    m = T(p["m_g"]).requires_grad_(True)
    coef = p["K_st"] if p["friction"] == "strickler" else p.get("f_dw", 0.0)
    K = T(coef).requires_grad_(True)
    _, _, _, zT = run(p, st, dts, A, m, K)
    L = torch.sum(T(lam_z).reshape(shape) * zT)
    gz, gh, gA, gm, gK = torch.autograd.grad(L, [z0, h0, A, m, K], allow_unused=True)
    z = lambda x: 0.0 if x is None else float(x)
    return dict(z=gz.numpy().reshape(w["z"].shape), h=gh.numpy().reshape(w["h"].shape),
                params=[z(gA), z(gm), z(gK)], zT=zT.detach().numpy().reshape(w["z"].shape))
