"""Seeded synthetic inputs for the Saint-Venant--Exner step.

This module holds only input recipes (initial and boundary data, physical
constants); none of the scheme's arithmetic.  Both the CUDA path and the CPU
oracle read the same arrays from here, and each maps the string-valued enums
(bedload law, friction law, boundary types) to its own codes.

Every generator returns ``dict(params=dict, h, hu, hv, z, nsteps)`` with
arrays of shape (ny, nx) in 2D and (nx,) in 1D (row-major, x fastest).

Recipes:
  * ``dune1d``      -- 1D Grass dune on a periodic 1000 m channel, a variant
    of the 1D dune test of Sec. 5.1 (free surface 2 m, q = 0.5 m^2/s).
  * ``dune2d``      -- 2D Gaussian dune in a 1000 x 500 m channel with inflow
    discharge and free outflow (shapes of the 2D bump test, Sec. 5.3),
    Grass + Strickler.
  * ``antidune2d``  -- supercritical channel 24 x 12 m (the length of the
    antidune test, Sec. 5.2), random bed perturbation, Meyer-Peter & Mueller
    + Darcy-Weisbach.
  * ``ensemble``    -- many independent ``dune2d``-type runs of uneven sizes
    and parameters.
  * ``adjoint_dune`` -- the dune physics in 2D on a periodic channel, the
    setting of the gradient (adjoint) runs.
  * ``paper_dune1d``, ``paper_antidune1d``, ``paper_bump2d`` -- the paper's
    own setups (Secs. 5.1--5.3) at a chosen resolution.
  * ``lake_at_rest``, ``thin_dam_break`` -- stress and property cases.
"""
from __future__ import annotations

import math

import numpy as np

G = 9.81

#: defaults of the numerical parameters every run carries
NUMERICS = dict(g=G, cfl=0.9, kappa_a=1.1, beta_min=0.01, gamma_z=2.0, newton_tol=1e-9, newton_maxit=30)


def base_params(**kw) -> dict:
    p = dict(
        dim=2, nx=1, ny=1, lx=1.0, ly=1.0,
        bedload="grass", A_g=1e-3, m_g=3.0, s=2.65, d_s=1e-3, tau_cr=0.05,
        friction="none", f_dw=0.0, K_st=0.0,
        bc=("periodic", "periodic", "free", "free"), q_in=0.0, h_in=0.0,
    )
    p.update(NUMERICS)
    p.update(kw)
    return p


def _centers(n: int, length: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def dune1d(nx: int = 1000, nsteps: int = 5000) -> dict:
    """1D dune, FP64: L = 1000 m, periodic, z = 0.1 + sin^2(pi (x-300)/200)
    on 300 < x < 500 else 0.1, free surface 2 m, hu = 0.5 m^2/s, Grass
    A_g = 1e-3, m_g = 3, CFL 0.9."""
    L = 1000.0
    x = _centers(nx, L)
    z = np.where((x > 300.0) & (x < 500.0), 0.1 + np.sin(np.pi * (x - 300.0) / 200.0) ** 2, 0.1)
    h = 2.0 - z
    hu = np.full(nx, 0.5)
    params = base_params(dim=1, nx=nx, ny=1, lx=L, ly=1.0, A_g=1e-3, m_g=3.0,
                         bc=("periodic", "periodic", "free", "free"))
    return dict(params=params, h=h, hu=hu, hv=None, z=z, nsteps=nsteps)


def dune2d(nx: int = 1024, ny: int = 512, seed: int = 0, nsteps: int = 2000, lx: float = 1000.0,
           ly: float = 500.0, A_g: float = 1e-3, m_g: float = 3.0, amp: tuple | None = None) -> dict:
    """2D dune, FP64: 1000 x 500 m, Gaussian bump z = 0.1 + A exp(-r^2/(2 50^2))
    with A ~ U[0.5, 1], centre x ~ U[250, 350], y ~ U[200, 300] (seeded),
    h = 2 - z, hu = 0.5, hv = 0; W inflow q = 0.5, E/S/N free; Grass m_g = 3,
    A_g = 1e-3, Strickler K = 40, CFL 0.9."""
    rng = np.random.default_rng(seed)
    lo, hi = amp if amp is not None else (0.5, 1.0)
    A = rng.uniform(lo, hi)
    xc = rng.uniform(0.25, 0.35) * lx
    yc = rng.uniform(0.4, 0.6) * ly
    sig = 50.0 * (lx / 1000.0)
    x = _centers(nx, lx)[None, :]
    y = _centers(ny, ly)[:, None]
    z = 0.1 + A * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2.0 * sig * sig))
    h = 2.0 - z
    hu = np.full((ny, nx), 0.5)
    hv = np.zeros((ny, nx))
    params = base_params(dim=2, nx=nx, ny=ny, lx=lx, ly=ly, A_g=A_g, m_g=m_g,
                         friction="strickler", K_st=40.0,
                         bc=("inflow_q", "free", "free", "free"), q_in=0.5)
    return dict(params=params, h=h, hu=hu, hv=hv, z=z, nsteps=nsteps)


def antidune2d(nx: int = 8192, ny: int = 4096, seed: int = 0, nsteps: int = 1000) -> dict:
    """2D antidune: 24 x 12 m, flat bed plus N(0, 0.01 m) per cell (seeded),
    h = h_in = 0.5 m, Froude ~ U[1.2, 1.5] (seeded), hu = q_in = Fr sqrt(g h) h;
    W supercritical inflow (h and q given), E/S/N free; Meyer-Peter & Mueller
    (s = 2.65, d_s = 1 mm, tau*_cr = 0.05) with Darcy-Weisbach f = 0.02."""
    rng = np.random.default_rng(seed)
    fr = rng.uniform(1.2, 1.5)
    h0 = 0.5
    q0 = fr * math.sqrt(G * h0) * h0
    z = rng.normal(0.0, 0.01, size=(ny, nx))
    h = np.full((ny, nx), h0)
    hu = np.full((ny, nx), q0)
    hv = np.zeros((ny, nx))
    params = base_params(dim=2, nx=nx, ny=ny, lx=24.0, ly=12.0, bedload="mpm", friction="darcy", f_dw=0.02,
                         bc=("inflow_qh", "free", "free", "free"), q_in=q0, h_in=h0)
    return dict(params=params, h=h, hu=hu, hv=hv, z=z, nsteps=nsteps)


def ensemble(nruns: int = 256, seed: int = 0, nsteps: int = 1000, nx_range=(128, 1024), ny_range=(64, 512)) -> list:
    """Batched ensemble: nruns independent 2D dune runs, Nx ~ U{128..1024},
    Ny ~ U{64..512}, A_g log-uniform in [1e-4, 1e-2], m_g in {1, 2, 3, 4},
    amplitude U[0.2, 1]; otherwise ``dune2d`` physics on 1000 x 500 m."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        A_g = float(10.0 ** rng.uniform(-4.0, -2.0))
        m_g = float(rng.integers(1, 5))
        amp = float(rng.uniform(0.2, 1.0))
        run = dune2d(nx=nx, ny=ny, seed=int(rng.integers(0, 2**31 - 1)), nsteps=nsteps, A_g=A_g, m_g=m_g,
                     amp=(amp, amp))
        runs.append(run)
    return runs


def adjoint_dune(nx: int = 2048, ny: int = 1024, nsteps: int = 4000, A_g: float = 1e-3, m_g: float = 3.0,
                 K_st: float = 40.0, shift: float = 0.0) -> dict:
    """Adjoint config: the 1D dune physics of ``dune1d`` in 2D on a periodic
    1000 x 500 m channel, z = 0.1 + sin^2(pi (x - 300 - shift)/200)
    sin^2(pi (y - 150)/200) on [300, 500] x [150, 350] (shifted in x by
    ``shift``), h = 2 - z, hu = 0.5, hv = 0, Grass A_g, m_g, Strickler K_st.
    The target bed of the misfit comes from a run with (1.1 A_g, m_g = 3.1,
    K_st = 36) and shift = 5 m."""
    lx, ly = 1000.0, 500.0
    x = _centers(nx, lx)[None, :] - shift
    y = _centers(ny, ly)[:, None]
    inside = (x >= 300.0) & (x <= 500.0) & (y >= 150.0) & (y <= 350.0)
    z = np.where(inside, 0.1 + np.sin(np.pi * (x - 300.0) / 200.0) ** 2 * np.sin(np.pi * (y - 150.0) / 200.0) ** 2,
                 0.1)
    h = 2.0 - z
    hu = np.full((ny, nx), 0.5)
    hv = np.zeros((ny, nx))
    params = base_params(dim=2, nx=nx, ny=ny, lx=lx, ly=ly, A_g=A_g, m_g=m_g, friction="strickler", K_st=K_st,
                         bc=("periodic",) * 4)
    return dict(params=params, h=h, hu=hu, hv=hv, z=z, nsteps=nsteps)


def paper_dune1d(nx: int = 2000, A_g: float = 1.0, m_g: float = 3.0) -> dict:
    """The 1D dune test of Sec. 5.1: L = 1000 m, z = 0.1 + sin^2((x-300) pi/200)
    on [300, 500], h = 10 - z, q = q0 = 10 m^2/s (inflow discharge at x = 0),
    Grass A_g = 1, m_g = 3.  Outflow: free."""
    L = 1000.0
    x = _centers(nx, L)
    z = np.where((x >= 300.0) & (x <= 500.0), 0.1 + np.sin((x - 300.0) * np.pi / 200.0) ** 2, 0.1)
    h = 10.0 - z
    hu = np.full(nx, 10.0)
    params = base_params(dim=1, nx=nx, ny=1, lx=L, A_g=A_g, m_g=m_g, bc=("inflow_q", "free", "free", "free"),
                         q_in=10.0)
    return dict(params=params, h=h, hu=hu, hv=None, z=z, nsteps=None)


def bernoulli_supercritical_depth(q0: float, head: float, z: np.ndarray, h_guess: float) -> np.ndarray:
    """Supercritical root h of q0^2/(2 g h^2) + h + z = head for every z
    (Newton from below the critical depth)."""
    hc = (q0 * q0 / G) ** (1.0 / 3.0)
    h = np.full_like(np.asarray(z, dtype=np.float64), min(h_guess, hc))
    for _ in range(200):
        f = q0 * q0 / (2.0 * G * h * h) + h + z - head
        df = 1.0 - q0 * q0 / (G * h ** 3)
        h_new = np.clip(h - f / df, 1e-6, hc)
        if np.max(np.abs(h_new - h)) < 1e-15:
            h = h_new
            break
        h = h_new
    return h


def paper_antidune1d(nx: int = 2400, bump: float = 0.2, A_g: float = 1e-3) -> dict:
    """The 1D antidune test of Sec. 5.2: L = 24 m, parabolic bump
    z = bump - 0.05 (x-10)^2 on [8, 12] (bump = 0.2 in the paper), q0 = 1.7,
    h from Bernoulli's law on the supercritical branch with h(0) = 0.5 m,
    Grass A_g = 1e-3, m_g = 3; supercritical inflow (h and q given), free
    outflow.  With bump = 0.2 the head at inflow is below the critical
    specific energy over the crest, so no supercritical profile exists there;
    callers pick a smaller bump (the depth is clipped at critical otherwise)."""
    L, q0, h0 = 24.0, 1.7, 0.5
    x = _centers(nx, L)
    z = np.where((x >= 8.0) & (x <= 12.0), np.maximum(bump - 0.05 * (x - 10.0) ** 2, 0.0), 0.0)
    head = q0 * q0 / (2.0 * G * h0 * h0) + h0 + 0.0
    h = bernoulli_supercritical_depth(q0, head, z, h0)
    hu = np.full(nx, q0)
    params = base_params(dim=1, nx=nx, ny=1, lx=L, A_g=A_g, m_g=3.0, bc=("inflow_qh", "free", "free", "free"),
                         q_in=q0, h_in=h0)
    return dict(params=params, h=h, hu=hu, hv=None, z=z, nsteps=None)


def paper_bump2d(nx: int = 4000, ny: int = 4000, A_g: float = 1.0) -> dict:
    """The 2D bump of Sec. 5.3: 1000 x 1000 m, z = 0.1 + sin^2(pi (x-300)/200)
    sin^2(pi (y-400)/200) on [300, 500] x [400, 600], h = 10 - z, q0 = 10 in
    x (upstream), free flow elsewhere, 2D Grass m_g = 3."""
    L = 1000.0
    x = _centers(nx, L)[None, :]
    y = _centers(ny, L)[:, None]
    inside = (x >= 300.0) & (x <= 500.0) & (y >= 400.0) & (y <= 600.0)
    z = np.where(inside, 0.1 + np.sin(np.pi * (x - 300.0) / 200.0) ** 2 * np.sin(np.pi * (y - 400.0) / 200.0) ** 2,
                 0.1)
    h = 10.0 - z
    hu = np.full((ny, nx), 10.0)
    hv = np.zeros((ny, nx))
    params = base_params(dim=2, nx=nx, ny=ny, lx=L, ly=L, A_g=A_g, m_g=3.0,
                         bc=("inflow_q", "free", "free", "free"), q_in=10.0)
    return dict(params=params, h=h, hu=hu, hv=hv, z=z, nsteps=None)


def lake_at_rest(nx: int = 100, dim: int = 1, ny: int = 1) -> dict:
    """Water at rest (h + z = 1, u = 0) over a smooth bump, rigid bed
    (A_g = 0), walls at both ends."""
    L = 10.0
    x = _centers(nx, L)
    zx = 0.2 * np.exp(-((x - 5.0) ** 2))
    if dim == 1:
        z = zx
        h = 1.0 - z
        return dict(params=base_params(dim=1, nx=nx, ny=1, lx=L, A_g=0.0, bc=("wall", "wall", "free", "free")),
                    h=h, hu=np.zeros(nx), hv=None, z=z, nsteps=None)
    z = np.repeat(zx[None, :], ny, axis=0)
    h = 1.0 - z
    return dict(params=base_params(dim=2, nx=nx, ny=ny, lx=L, ly=L * ny / nx, A_g=0.0,
                                   bc=("wall", "wall", "wall", "wall")),
                h=h, hu=np.zeros((ny, nx)), hv=np.zeros((ny, nx)), z=z, nsteps=None)


def thin_dam_break(nx: int = 200, h_thin: float = 1e-3) -> dict:
    """Dam break from 1 m onto a thin layer (h_thin) over a flat bed, walls,
    Grass A_g = 1e-3, CFL 0.5: the positivity stress case."""
    L = 10.0
    x = _centers(nx, L)
    h = np.where(x < 5.0, 1.0, h_thin)
    z = np.zeros(nx)
    params = base_params(dim=1, nx=nx, ny=1, lx=L, A_g=1e-3, cfl=0.5, bc=("wall", "wall", "free", "free"))
    return dict(params=params, h=h, hu=np.zeros(nx), hv=None, z=z, nsteps=None)


def bed_step(nx: int = 100, dim: int = 1, ny: int = 1, step: float = 0.4, q: float = 0.5,
             A_g: float = 1e-3) -> dict:
    """Flow of discharge q over a bed step of height `step` at mid-channel
    (10 m long, free surface at 1.2 m): a step of about a third of the depth,
    where the bed-jump bound of the celerities sets a (the stronger bound of
    Sec. 3, reading R1).  Inflow q on the west side, free elsewhere.  In 2D
    the step line is oblique (x = 5 m + 0.5 (y - ly/2)), so x- and
    y-interfaces both cross it."""
    L = 10.0
    x = _centers(nx, L)
    if dim == 1:
        z = np.where(x > 0.5 * L, step, 0.0)
        params = base_params(dim=1, nx=nx, ny=1, lx=L, A_g=A_g, q_in=q, bc=("inflow_q", "free", "free", "free"))
        return dict(params=params, h=1.2 - z, hu=np.full(nx, q), hv=None, z=z, nsteps=None)
    ly = L * ny / nx
    y = _centers(ny, ly)
    X, Y = np.meshgrid(x, y)
    z = np.where(X > 0.5 * L + 0.5 * (Y - 0.5 * ly), step, 0.0)
    params = base_params(dim=2, nx=nx, ny=ny, lx=L, ly=ly, A_g=A_g, q_in=q, bc=("inflow_q", "free", "free", "free"))
    return dict(params=params, h=1.2 - z, hu=np.full_like(z, q), hv=np.zeros_like(z), z=z, nsteps=None)


def colliding_streams(nx: int = 200, dim: int = 1, ny: int = 1, h0: float = 0.1, u0: float = 3.0,
                      A_g: float = 1e-2, m_g: float = 3.0, ymod: float = 0.0) -> dict:
    """Two supercritical streams (depth h0, speeds +u0 and -u0, Froude
    u0 / sqrt(g h0)) meeting at the middle of a 10 m walled channel over a
    flat mobile bed (Grass law): the strong compression where the
    relaxation solver halves Newton steps and, at the first steps, needs
    celerities above its default bounds.  In 2D the depth varies across the
    channel by the relative amplitude ymod (one sine period over ly), walls
    on all sides."""
    L = 10.0
    x = _centers(nx, L)
    if dim == 1:
        h = np.full(nx, h0)
        hu = np.where(x < 0.5 * L, h0 * u0, -h0 * u0)
        params = base_params(dim=1, nx=nx, ny=1, lx=L, A_g=A_g, m_g=m_g, bc=("wall", "wall", "free", "free"))
        return dict(params=params, h=h, hu=hu, hv=None, z=np.zeros(nx), nsteps=None)
    ly = L * ny / nx
    y = _centers(ny, ly)
    X, Y = np.meshgrid(x, y)
    h = h0 * (1.0 + ymod * np.sin(2.0 * np.pi * Y / ly))
    hu = np.where(X < 0.5 * L, 1.0, -1.0) * h * u0
    params = base_params(dim=2, nx=nx, ny=ny, lx=L, ly=ly, A_g=A_g, m_g=m_g,
                         bc=("wall", "wall", "wall", "wall"))
    return dict(params=params, h=h, hu=hu, hv=np.zeros_like(h), z=np.zeros_like(h), nsteps=None)


def random_smooth(nx: int, ny: int, seed: int, dim: int = 2, bc=("periodic", "periodic", "periodic", "periodic"),
                  **kw) -> dict:
    """Smooth random state (h in [0.8, 1.2], |u| < 0.5, z in [0, 0.2]) as a
    sum of a few seeded Fourier modes; periodic-compatible."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny if dim == 2 else np.zeros(1)
    X, Y = np.meshgrid(x, y)

    def field(amp):
        f = np.zeros_like(X)
        for _ in range(3):
            kx, ky = rng.integers(1, 4), (rng.integers(0, 3) if dim == 2 else 0)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.uniform(-amp, amp) * np.sin(2 * np.pi * (kx * X + ky * Y) + ph)
        return f

    h = 1.0 + field(0.07)
    u = 0.3 + field(0.05)
    v = field(0.05) if dim == 2 else np.zeros_like(X)
    z = 0.1 + field(0.03)
    params = base_params(dim=dim, nx=nx, ny=ny if dim == 2 else 1, lx=float(nx), ly=float(ny), bc=bc, **kw)
    if dim == 1:
        return dict(params=params, h=h[0], hu=(h * u)[0], hv=None, z=z[0], nsteps=None)
    return dict(params=params, h=h, hu=h * u, hv=h * v, z=z, nsteps=None)
