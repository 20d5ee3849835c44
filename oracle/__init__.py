"""FP64 CPU oracle for the Saint-Venant--Exner relaxation step.

TEST INFRASTRUCTURE ONLY: the reference the CUDA path is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1307_0491_gb300``) and never imports it.

The arithmetic lives in ``sve_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module only compiles it and marshals arrays
through ``ctypes``.  Every function of the C file cites the passage of the
paper (arXiv:1307.0491) it follows.

Parity status per function (what pins it, see ``tests/test_oracle_pins.py``):
  * ``riemann``      -- pinned: Riemann invariants across each wave,
    Rankine--Hugoniot relations of the conservative rows, the generalised
    momentum jump at the sediment waves, wave order / positivity, reduction
    to the Suliciu solver at A_g = 0 on a flat bed, an independent 50-digit
    solve of the invariant system.
  * ``run`` / ``cfl`` -- pinned: mass conservation on periodic and walled
    domains, positivity, y-invariant 2D == 1D, an independent 50-digit
    single step on 4--8 cell grids, migration direction of dunes (Fr < 1)
    and antidunes (Fr > 1), lack of well-balancing.
  * ``cell_project`` -- pinned: closed forms of the Grass and MPM laws and
    finite-difference derivatives.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sve_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsve_oracle.so")

GRASS, MPM, FLVB, NIELSEN, RIBBERINK, CAMENEN = 0, 1, 2, 3, 4, 5
FRIC_NONE, FRIC_DARCY, FRIC_STRICKLER = 0, 1, 2
BC_PERIODIC, BC_FREE, BC_INFLOW_Q, BC_INFLOW_QH, BC_WALL = 0, 1, 2, 3, 4

ERRORS = {0: "ok", -1: "arg", -4: "neg_depth", -5: "riemann", -6: "nan", -7: "dt"}


def build_oracle(force: bool = False, src: str | None = None, out: str | None = None) -> str:
    """Compile the C oracle into a shared library and return its path."""
    src = src or _SRC
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["cc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("g", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bedload", ctypes.c_int),
        ("A_g", ctypes.c_double), ("m_g", ctypes.c_double),
        ("s", ctypes.c_double), ("d_s", ctypes.c_double), ("tau_cr", ctypes.c_double),
        ("friction", ctypes.c_int),
        ("f_dw", ctypes.c_double), ("K_st", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("q_in", ctypes.c_double), ("h_in", ctypes.c_double),
        ("kappa_a", ctypes.c_double), ("beta_min", ctypes.c_double), ("gamma_z", ctypes.c_double),
        ("newton_tol", ctypes.c_double),
        ("newton_maxit", ctypes.c_int),
    ]


class _RiemannOut(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("K", ctypes.c_double),
        ("lam", ctypes.c_double * 5),
        ("tau", ctypes.c_double * 6), ("u", ctypes.c_double * 6), ("v", ctypes.c_double * 6),
        ("Z", ctypes.c_double * 6), ("Pi", ctypes.c_double * 6), ("Om", ctypes.c_double * 6),
        ("Am", ctypes.c_double * 4), ("Ap", ctypes.c_double * 4),
        ("iters", ctypes.c_int), ("status", ctypes.c_int),
        ("halvings", ctypes.c_int), ("raised", ctypes.c_int), ("retries", ctypes.c_int),
    ]


@dataclass
class Params:
    """Physical and numerical parameters of one run (oracle-side mirror)."""

    dim: int = 2
    nx: int = 16
    ny: int = 1
    lx: float = 1.0
    ly: float = 1.0
    g: float = 9.81
    cfl: float = 0.9
    bedload: int = GRASS
    A_g: float = 1e-3
    m_g: float = 3.0
    s: float = 2.65
    d_s: float = 1e-3
    tau_cr: float = 0.05
    friction: int = FRIC_NONE
    f_dw: float = 0.0
    K_st: float = 0.0
    bc: tuple = (BC_PERIODIC, BC_PERIODIC, BC_FREE, BC_FREE)
    q_in: float = 0.0
    h_in: float = 0.0
    kappa_a: float = 1.1
    beta_min: float = 0.01
    gamma_z: float = 2.0
    newton_tol: float = 1e-9
    newton_maxit: int = 30

    def to_c(self) -> _Params:
        p = _Params()
        for name, _ in _Params._fields_:
            if name == "bc":
                p.bc = (ctypes.c_int * 4)(*[int(b) for b in self.bc])
            else:
                setattr(p, name, getattr(self, name))
        return p

    @staticmethod
    def from_workload(d: dict) -> "Params":
        """Map a workload parameter dict (string-valued enums) to the
        oracle's own codes."""
        bedload = {"grass": GRASS, "mpm": MPM, "flvb": FLVB, "nielsen": NIELSEN, "ribberink": RIBBERINK,
                   "camenen": CAMENEN}
        friction = {"none": FRIC_NONE, "darcy": FRIC_DARCY, "strickler": FRIC_STRICKLER}
        bc = {"periodic": BC_PERIODIC, "free": BC_FREE, "inflow_q": BC_INFLOW_Q, "inflow_qh": BC_INFLOW_QH,
              "wall": BC_WALL}
        keys = {f for f in Params.__dataclass_fields__}
        kw = {k: v for k, v in d.items() if k in keys}
        if isinstance(kw.get("bedload"), str):
            kw["bedload"] = bedload[kw["bedload"]]
        if isinstance(kw.get("friction"), str):
            kw["friction"] = friction[kw["friction"]]
        if "bc" in kw:
            kw["bc"] = tuple(bc[b] if isinstance(b, str) else int(b) for b in kw["bc"])
        return Params(**kw)


class OracleError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"oracle {where}: status {code} ({ERRORS.get(code, '?')})")
        self.code = code


class Oracle:
    """ctypes handle on one compiled oracle library (the default one, or a
    variant compiled from another source file, e.g. a planted mistake)."""

    def __init__(self, lib_path: str | None = None):
        path = lib_path or build_oracle()
        self.lib = ctypes.CDLL(path)
        L = self.lib
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_riemann.argtypes = [ctypes.POINTER(_Params), dp, dp, ctypes.POINTER(_RiemannOut)]
        L.orc_riemann.restype = ctypes.c_int
        L.orc_cell_project.argtypes = [ctypes.POINTER(_Params), dp, dp]
        L.orc_cell_project.restype = ctypes.c_int
        L.orc_cfl.argtypes = [ctypes.POINTER(_Params), dp, dp, dp, dp, dp]
        L.orc_cfl.restype = ctypes.c_int
        L.orc_run.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, dp, dp, dp, dp, dp, dp, dp, dp,
                              ctypes.POINTER(ctypes.c_int)]
        L.orc_run.restype = ctypes.c_int
        L.orc_split_run.argtypes = L.orc_run.argtypes
        L.orc_split_run.restype = ctypes.c_int
        blk = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        L.orc_block_ghost.argtypes = blk + [ctypes.c_int]
        L.orc_block_solve.argtypes = blk + [dp, dp]
        L.orc_block_update.argtypes = blk + [dp, ctypes.c_double]
        for name in ("orc_block_ghost", "orc_block_solve", "orc_block_update"):
            getattr(L, name).restype = ctypes.c_int
        L.orc_block_dt.argtypes = [ctypes.POINTER(_Params), ctypes.c_double, ctypes.c_double, dp]
        L.orc_block_dt.restype = ctypes.c_int
        assert L.orc_sizeof_params() == ctypes.sizeof(_Params), "oracle params struct mismatch"
        assert L.orc_sizeof_riemann_out() == ctypes.sizeof(_RiemannOut), "oracle riemann struct mismatch"

    # -- single interface ------------------------------------------------
    def riemann(self, p: Params, Lc, Rc) -> dict:
        """Solve one interface; Lc, Rc = (H, H un, H ut, Z) in the normal frame."""
        lc = (ctypes.c_double * 4)(*[float(x) for x in Lc])
        rc = (ctypes.c_double * 4)(*[float(x) for x in Rc])
        out = _RiemannOut()
        cp = p.to_c()
        st = self.lib.orc_riemann(ctypes.byref(cp), lc, rc, ctypes.byref(out))
        res = {
            "status": st, "iters": out.iters, "halvings": out.halvings, "raised": out.raised,
            "retries": out.retries, "a": out.a, "b": out.b, "K": out.K,
            "lam": np.array(out.lam[:]),
            "tau": np.array(out.tau[:]), "u": np.array(out.u[:]), "v": np.array(out.v[:]),
            "Z": np.array(out.Z[:]), "Pi": np.array(out.Pi[:]), "Om": np.array(out.Om[:]),
            "Am": np.array(out.Am[:]), "Ap": np.array(out.Ap[:]),
        }
        return res

    def cell_project(self, p: Params, c) -> dict:
        cc = (ctypes.c_double * 4)(*[float(x) for x in c])
        out = (ctypes.c_double * 8)()
        cp = p.to_c()
        st = self.lib.orc_cell_project(ctypes.byref(cp), cc, out)
        if st:
            raise OracleError(st, "cell_project")
        keys = ("tau", "un", "ut", "Pi", "Om", "dOm", "ca", "cb")
        return dict(zip(keys, out[:]))

    # -- whole grid ------------------------------------------------------
    @staticmethod
    def _arr(x, n):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1)).copy()
        if a.size != n:
            raise ValueError(f"expected {n} values, got {a.size}")
        return a

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None

    def cfl(self, p: Params, h, hu, hv, z) -> float:
        n = p.nx * p.ny
        h, hu, z = self._arr(h, n), self._arr(hu, n), self._arr(z, n)
        hv = self._arr(hv, n) if (p.dim == 2) else None
        dt = ctypes.c_double(0.0)
        cp = p.to_c()
        st = self.lib.orc_cfl(ctypes.byref(cp), self._ptr(h), self._ptr(hu), self._ptr(hv), self._ptr(z),
                              ctypes.byref(dt))
        if st:
            raise OracleError(st, "cfl")
        return dt.value

    def run(self, p: Params, nsteps: int, h, hu, hv, z, dts=None, t0: float = 0.0, check: bool = True,
            split: bool = False) -> dict:
        """Advance nsteps steps (CFL steps, or the given fixed steps dts);
        split: the splitting scheme (shallow-water step, then the Exner
        update of the bed: reading R13 of sve_oracle.c) instead of the coupled
        step.

        Returns dict(h, hu, hv, z, t, dts, diag, status, done) with arrays
        shaped (ny, nx) (1D: (nx,))."""
        n = p.nx * p.ny
        h, hu, z = self._arr(h, n), self._arr(hu, n), self._arr(z, n)
        hv = self._arr(hv, n) if p.dim == 2 else None
        fixed = None
        if dts is not None:
            fixed = np.ascontiguousarray(np.asarray(dts, dtype=np.float64).reshape(-1))
            if fixed.size < nsteps:
                raise ValueError("need one dt per step")
        t = ctypes.c_double(t0)
        dts_out = np.zeros(max(nsteps, 1))
        diag = np.zeros(2 * max(nsteps, 1))
        done = ctypes.c_int(0)
        cp = p.to_c()
        fn = self.lib.orc_split_run if split else self.lib.orc_run
        st = fn(ctypes.byref(cp), int(nsteps), self._ptr(fixed), self._ptr(h), self._ptr(hu), self._ptr(hv),
                self._ptr(z), ctypes.byref(t), self._ptr(dts_out), self._ptr(diag), ctypes.byref(done))
        if st and check:
            raise OracleError(st, f"run (after {done.value} steps)")
        shape = (p.ny, p.nx) if p.dim == 2 else (p.nx,)
        return {
            "h": h.reshape(shape), "hu": hu.reshape(shape), "hv": hv.reshape(shape) if hv is not None else None,
            "z": z.reshape(shape), "t": t.value, "dts": dts_out[:nsteps], "diag": diag[: 2 * nsteps].reshape(-1, 2),
            "status": st, "done": done.value,
        }


class Block:
    """One padded block (nxl + 2) x (nyl + 2) of a domain decomposition of
    the grid of ``params`` (whose nx, ny are the whole grid's sizes)."""

    def __init__(self, orc: "Oracle", p: Params, nxl: int, nyl: int):
        self.orc, self.p, self.cp = orc, p, p.to_c()
        self.nxl, self.nyl = nxl, nyl
        self.f = {k: np.zeros((nyl + 2, nxl + 2)) for k in ("h", "hu", "hv", "z")}
        self.work = np.zeros(4 * nxl * nyl)  # net fluctuations of the last solve
        self.solved = False

    def set_interior(self, h, hu, hv, z):
        for k, a in zip(("h", "hu", "hv", "z"), (h, hu, hv, z)):
            self.f[k][1:-1, 1:-1] = np.asarray(a).reshape(self.nyl, self.nxl)

    def interior(self, k):
        return self.f[k][1:-1, 1:-1]

    def _ptrs(self):
        return [self.f[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for k in ("h", "hu", "hv", "z")]

    def ghost(self, side: int):
        st = self.orc.lib.orc_block_ghost(ctypes.byref(self.cp), self.nxl, self.nyl, *self._ptrs(), int(side))
        if st:
            raise OracleError(st, "block_ghost")

    def speeds(self):
        """Solve every interface of the block (ghosts filled), keep the net
        fluctuations for ``advance`` and return the extreme speeds."""
        S = (ctypes.c_double * 2)()
        wp = self.work.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st = self.orc.lib.orc_block_solve(ctypes.byref(self.cp), self.nxl, self.nyl, *self._ptrs(), wp, S)
        if st:
            raise OracleError(st, "block_solve")
        self.solved = True
        return S[0], S[1]

    def dt(self, Sx: float, Sy: float) -> float:
        d = ctypes.c_double(0.0)
        st = self.orc.lib.orc_block_dt(ctypes.byref(self.cp), Sx, Sy, ctypes.byref(d))
        if st:
            raise OracleError(st, "block_dt")
        return d.value

    def advance(self, dt: float):
        """Step dt from the fluctuations of the preceding ``speeds`` call."""
        if not self.solved:
            raise RuntimeError("Block.advance needs the solve of Block.speeds on the same state")
        wp = self.work.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st = self.orc.lib.orc_block_update(ctypes.byref(self.cp), self.nxl, self.nyl, *self._ptrs(), wp,
                                           float(dt))
        self.solved = False
        if st:
            raise OracleError(st, "block_update")


_DEFAULT: Oracle | None = None


def get() -> Oracle:
    """The oracle compiled from ``sve_oracle.c`` (built on first use)."""
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT
