"""Independent restatements used to pin the oracle (test code only).

Nothing here imports the oracle.  Each routine restates a piece of the
method from its definition in a different form than ``oracle/sve_oracle.c``:

* ``closure``            -- Grass (Eq. bedload Grass) and the Shields-
                            parameter laws (Eqs. MPM, FLVB, Nielsen, Ribberink,
                            Camenen with the non-dimensional form of Sec. 2)
                            in closed form (``qstar``: the laws' rates).
* ``celerities``         -- the bounds of Eq. (ab) with reading R1 (incl. the
                            bed-step term gamma_z).
* ``suliciu_fluct``      -- the textbook Suliciu relaxation solver for shallow
                            water (Bouchut 2004, Sec. 2.4, constant a), which
                            is the fluid part of the relaxation model (Sec. 3,
                            first property of the relaxation model).
* ``mp_riemann``         -- the relaxation Riemann problem solved as the
                            4-unknown system of contact conditions in 50-digit
                            arithmetic (mpmath), instead of the scalar Newton.
* ``mp_step``            -- one whole step (ghosts, CFL, fluxes, update,
                            friction) built on ``mp_riemann``.
"""
from __future__ import annotations

import math

G = 9.81


def closure(p: dict, H, un, ut, lib=math):
    """(Q, dQ/dun) of the bedload law for a cell; p uses workload keys."""
    speed2 = un * un + ut * ut
    if p["bedload"] == "grass":
        A, m = p["A_g"], p["m_g"]
        if speed2 == 0:
            return 0 * H, (A if m == 1 else 0 * H)
        sp = lib.sqrt(speed2)
        Q = A * un * sp ** (m - 1)
        dQ = A * (sp ** (m - 1) + (m - 1) * un * un * sp ** (m - 3))
        return Q, dQ
    sm1 = p["s"] - 1
    g = p["g"]
    if p["friction"] == "darcy":
        alpha = p["f_dw"] / (8 * g * sm1 * p["d_s"])
    else:
        n = 1 / p["K_st"]
        alpha = n * n / (sm1 * p["d_s"] * H ** (lib.mpf(1) / 3 if lib is not math else 1.0 / 3.0))
    q, dq = qstar(p["bedload"], alpha * speed2, p["tau_cr"], lib)
    if speed2 == 0 or (q == 0 and dq == 0):
        return 0 * H, 0 * H
    sp = lib.sqrt(speed2)
    C = lib.sqrt(sm1 * g * p["d_s"] ** 3)
    Q = C * q * un / sp
    dQ = C * (2 * alpha * dq * un * un / sp + q * ut * ut / sp ** 3)
    return Q, dQ


def qstar(law: str, ts, tcr, lib=math):
    """(q*, dq*/dtau*) of the Shields-parameter laws listed in Sec. 2 (Eqs.
    MPM, FLVB, Nielsen, Ribberink, Camenen); the derivative from each law's
    logarithmic derivative."""
    if law == "camenen":
        if ts <= 0:
            return 0 * ts, 0 * ts
        q = 12 * ts * lib.sqrt(ts) * lib.exp(-4.5 * tcr / ts)
        return q, q * (1.5 / ts + 4.5 * tcr / (ts * ts))
    x = ts - tcr
    if x <= 0:
        return 0 * ts, 0 * ts
    if law == "nielsen":
        q = 12 * lib.sqrt(ts) * x
        return q, q * (1 / (2 * ts) + 1 / x)
    K, pw = {"mpm": (8, 1.5), "flvb": (5.7, 1.5), "ribberink": (11, 1.65)}[law]
    q = K * x ** pw
    return q, q * pw / x


def celerities(p: dict, L, R, lib=math):
    """(a, b) of reading R1 for conserved states L, R = (H, H un, H ut, Z)."""
    g = p["g"]
    vals = []
    for c in (L, R):
        H = c[0]
        un, ut = c[1] / H, c[2] / H
        _, dQ = closure(p, H, un, ut, lib)
        vals.append((H * lib.sqrt(g * H), lib.sqrt(c[1] * c[1] + g * H * H * dQ)))
    a0 = max(vals[0][0], vals[1][0])
    b0 = max(vals[0][1], vals[1][1])
    a = p["kappa_a"] * max(a0, b0)
    b = max(b0, p["beta_min"] * a0)
    # K tau_min^2 >= gamma_z |dZ|  <=>  a^2 >= b^2 + 2 g gamma_z |dZ| Hmax^2
    Hmax = max(L[0], R[0])
    a = max(a, lib.sqrt(b * b + 2 * g * p["gamma_z"] * abs(R[3] - L[3]) * Hmax * Hmax))
    return a, b


def suliciu_fluct(p: dict, L, R):
    """Fluctuations (A-, A+) of (H, Hu, Hv) of the Suliciu solver with the
    constant a of reading R1, from interface fluxes: A- = F(0) - F_L,
    A+ = F_R - F(0)."""
    g = p["g"]
    a, _ = celerities(p, L, R)
    HL, HR = L[0], R[0]
    tL, tR = 1 / HL, 1 / HR
    uL, uR = L[1] / HL, R[1] / HR
    vL, vR = L[2] / HL, R[2] / HR
    PL, PR = g * HL * HL / 2, g * HR * HR / 2
    us = (uL + uR) / 2 - (PR - PL) / (2 * a)
    Ps = (PL + PR) / 2 - a * (uR - uL) / 2
    tLs = tL + (us - uL) / a
    tRs = tR - (us - uR) / a

    def flux(H, u, v, P):
        return (H * u, H * u * u + P, H * u * v)

    if uL - a * tL >= 0:
        F0 = flux(HL, uL, vL, PL)
    elif us >= 0:
        F0 = flux(1 / tLs, us, vL, Ps)
    elif uR + a * tR >= 0:
        F0 = flux(1 / tRs, us, vR, Ps)
    else:
        F0 = flux(HR, uR, vR, PR)
    FL = flux(HL, uL, vL, PL)
    FR = flux(HR, uR, vR, PR)
    Am = [F0[k] - FL[k] for k in range(3)]
    Ap = [FR[k] - F0[k] for k in range(3)]
    return Am, Ap, a


# ---------------------------------------------------------------------------
# 50-digit solve of the relaxation Riemann problem

def mp_riemann(p: dict, L, R, dps: int = 50, start=None, ab=None):
    """Relaxation Riemann problem as four contact conditions in the four
    unknown specific volumes (tau1..tau4), every other quantity written from
    the Riemann invariants of the a- and b-waves (Eqs. relaxh--relaxqs).
    The multidimensional root search starts from (tauL, tauL, tauR, tauR),
    or from ``start`` (four specific volumes) where the system has several
    roots and the one near a given point is wanted.  The celerities are those
    of reading R1, or ``ab`` = (a, b) where a solve used others.
    Returns dict(lam[5], U[6][4], a, b) in mpmath numbers."""
    import mpmath as mp

    mp.mp.dps = dps
    g = mp.mpf(p["g"])
    q = dict(p)
    q["g"] = g
    L = [mp.mpf(x) for x in L]
    R = [mp.mpf(x) for x in R]
    a, b = celerities(q, L, R, lib=mp) if ab is None else (mp.mpf(ab[0]), mp.mpf(ab[1]))
    K = (a * a - b * b) / (2 * g)
    HL, HR = L[0], R[0]
    tL, tR = 1 / HL, 1 / HR
    uL, uR = L[1] / HL, R[1] / HR
    vL, vR = L[2] / HL, R[2] / HR
    ZL, ZR = L[3], R[3]
    PL, PR = g * HL * HL / 2, g * HR * HR / 2
    OL, _ = closure(q, HL, uL, vL, lib=mp)
    OR, _ = closure(q, HR, uR, vR, lib=mp)

    def states(t1, t2, t3, t4):
        u1 = uL + a * (t1 - tL)           # u - a tau invariant across lambda1
        u2 = u1 + b * (t2 - t1)           # u - b tau invariant across lambda2
        u4 = uR - a * (t4 - tR)           # u + a tau invariant across lambda5
        u3 = u4 + b * (t4 - t3)           # u + b tau invariant across lambda4
        P2 = PL + a * a * (tL - t2)       # Pi + a^2 tau invariant (all but contact)
        P3 = PR + a * a * (tR - t3)
        Z2 = ZL + K * (t2 * t2 - t1 * t1)  # Z - K tau^2 invariant across b-waves
        Z3 = ZR + K * (t3 * t3 - t4 * t4)
        l2 = u1 - b * t1
        l4 = u4 + b * t4
        O2 = OL + l2 * (Z2 - ZL)          # Omega - lambda Z invariant across b-waves
        O3 = OR - l4 * (ZR - Z3)
        return u1, u2, u3, u4, P2, P3, Z2, Z3, l2, l4, O2, O3

    def eqs(t1, t2, t3, t4):
        u1, u2, u3, u4, P2, P3, Z2, Z3, l2, l4, O2, O3 = states(t1, t2, t3, t4)
        return [u2 - u3, P2 - P3, Z2 - Z3, O2 - O3]

    if list(L) == list(R):
        sol = [tL, tL, tR, tR]
    else:
        x0 = (tL, tL, tR, tR) if start is None else tuple(mp.mpf(x) for x in start)
        sol = mp.findroot(eqs, x0, tol=mp.mpf(10) ** (-(dps - 8)), maxsteps=200)
        sol = [sol[i] for i in range(4)]
    t1, t2, t3, t4 = sol
    u1, u2, u3, u4, P2, P3, Z2, Z3, l2, l4, O2, O3 = states(t1, t2, t3, t4)
    lam = [uL - a * tL, l2, u2, l4, uR + a * tR]
    taus = [t1, t2, t3, t4]
    us = [u1, u2, u3, u4]
    vs = [vL, vL, vR, vR]
    Zs = [ZL, Z2, Z3, ZR]
    U = [list(L)]
    for k in range(4):
        H = 1 / taus[k]
        U.append([H, H * us[k], H * vs[k], Zs[k]])
    U.append(list(R))
    return dict(lam=lam, U=U, a=a, b=b, tau=taus)


def mp_fluct(p: dict, L, R, dps: int = 50, start=None, ab=None):
    import mpmath as mp

    r = mp_riemann(p, L, R, dps, start, ab)
    Am = [mp.mpf(0)] * 4
    Ap = [mp.mpf(0)] * 4
    for k in range(5):
        lk = r["lam"][k]
        for c in range(4):
            j = r["U"][k + 1][c] - r["U"][k][c]
            if lk < 0:
                Am[c] += lk * j
            elif lk > 0:
                Ap[c] += lk * j
    return Am, Ap, r


def _ghost(p, side, s):
    """Ghost state from the adjacent state s = [H, Hu, Hv, Z] (reading R7)."""
    t = p["bc"][side]
    out = list(s)
    normal = 1 if side < 2 else 2
    tangent = 2 if side < 2 else 1
    inward = 1 if side in (0, 2) else -1
    if t == "inflow_q":
        out[normal] = inward * p["q_in"]
        out[tangent] = 0
    elif t == "inflow_qh":
        out[0] = p["h_in"]
        out[normal] = inward * p["q_in"]
        out[tangent] = 0
    elif t == "wall":
        out[normal] = -s[normal]
    return out


def mp_step(p: dict, h, hu, hv, z, dt=None, dps: int = 50):
    """One step in 50-digit arithmetic.  h, hu, hv, z: nested lists [ny][nx]
    (1D: ny = 1, hv ignored).  Returns (new state lists, dt)."""
    import mpmath as mp

    mp.mp.dps = dps
    dim, nx, ny = p["dim"], p["nx"], p["ny"]
    g = mp.mpf(p["g"])
    q = dict(p)
    q["g"] = g
    cell = lambda j, i: [mp.mpf(h[j][i]), mp.mpf(hu[j][i]), mp.mpf(hv[j][i]) if dim == 2 else mp.mpf(0),
                         mp.mpf(z[j][i])]

    def get(j, i):
        if 0 <= i < nx and 0 <= j < ny:
            return cell(j, i)
        if i < 0:
            return _ghost(q, 0, cell(j, nx - 1 if p["bc"][0] == "periodic" else 0))
        if i >= nx:
            return _ghost(q, 1, cell(j, 0 if p["bc"][1] == "periodic" else nx - 1))
        if j < 0:
            return _ghost(q, 2, cell(ny - 1 if p["bc"][2] == "periodic" else 0, i))
        return _ghost(q, 3, cell(0 if p["bc"][3] == "periodic" else ny - 1, i))

    rot = lambda s: [s[0], s[2], s[1], s[3]]  # y-normal frame
    dx = mp.mpf(p["lx"]) / nx
    dy = mp.mpf(p["ly"]) / ny if dim == 2 else mp.mpf(1)
    xint = {}
    yint = {}
    Sx = Sy = mp.mpf(0)
    for j in range(ny):
        for i in range(nx + 1):
            Lc, Rc = get(j, i - 1), get(j, i)
            a, _ = celerities(q, Lc, Rc, lib=mp)
            Sx = max(Sx, abs(Lc[1] / Lc[0] - a / Lc[0]), abs(Rc[1] / Rc[0] + a / Rc[0]))
            xint[(j, i)] = (Lc, Rc)
    if dim == 2:
        for j in range(ny + 1):
            for i in range(nx):
                Lc, Rc = rot(get(j - 1, i)), rot(get(j, i))
                a, _ = celerities(q, Lc, Rc, lib=mp)
                Sy = max(Sy, abs(Lc[1] / Lc[0] - a / Lc[0]), abs(Rc[1] / Rc[0] + a / Rc[0]))
                yint[(j, i)] = (Lc, Rc)
    if dt is None:
        dt = p["cfl"] * dx / Sx if dim == 1 else p["cfl"] / (Sx / dx + Sy / dy)
    else:
        dt = mp.mpf(dt)
    fx = {k: mp_fluct(q, *v, dps=dps) for k, v in xint.items()}
    fy = {k: mp_fluct(q, *v, dps=dps) for k, v in yint.items()}
    out = [[None] * nx for _ in range(ny)]
    for j in range(ny):
        for i in range(nx):
            U = cell(j, i)
            Ap = fx[(j, i)][1]
            Am = fx[(j, i + 1)][0]
            new = [U[c] - dt / dx * (Ap[c] + Am[c]) for c in range(4)]
            if dim == 2:
                Bp = rot(fy[(j, i)][1])
                Bm = rot(fy[(j + 1, i)][0])
                new = [new[c] - dt / dy * (Bp[c] + Bm[c]) for c in range(4)]
            if p["friction"] != "none":
                Hn = new[0]
                qn = mp.sqrt(new[1] ** 2 + new[2] ** 2)
                if p["friction"] == "darcy":
                    C = p["f_dw"] / (8 * Hn * Hn)
                else:
                    C = g / (mp.mpf(p["K_st"]) ** 2 * Hn ** (mp.mpf(7) / 3))
                new[1] = new[1] / (1 + dt * C * qn)
                new[2] = new[2] / (1 + dt * C * qn)
            out[j][i] = new
    return out, dt
