"""Python binding of libsve (include/sve.h): argument marshalling only.

The functions ``sve_*`` below have the names and arguments of the C ABI; all
work of a step runs in the library's CUDA kernels.  ``Solver`` is a thin
convenience wrapper that maps a workload parameter dict (string-valued
enums) to ``sve_config`` and moves numpy arrays or torch tensors in and out.

The library must have been built (``paper_1307_0491_gb300.build.build()``);
there is no fallback: loading fails loudly when ``libsve.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SVE_OK = 0
SVE_ERR_ARG, SVE_ERR_CUDA, SVE_ERR_OOM = -1, -2, -3
SVE_ERR_NEG_DEPTH, SVE_ERR_RIEMANN, SVE_ERR_NAN, SVE_ERR_DT, SVE_ERR_STATE = -4, -5, -6, -7, -8
SVE_ERR_NOALLOC_SIZE = -9
SVE_ERR_SYNC = -10
SVE_NOALLOC_SCRATCH_BYTES = 8 << 20
SVE_FP64, SVE_FP32 = 0, 1
SVE_SCHEME_COUPLED, SVE_SCHEME_SPLIT = 0, 1
SVE_GRASS, SVE_MPM, SVE_FLVB, SVE_NIELSEN, SVE_RIBBERINK, SVE_CAMENEN = 0, 1, 2, 3, 4, 5
SVE_FRIC_NONE, SVE_FRIC_DARCY, SVE_FRIC_STRICKLER = 0, 1, 2
SVE_BC_PERIODIC, SVE_BC_FREE, SVE_BC_INFLOW_Q, SVE_BC_INFLOW_QH, SVE_BC_WALL, SVE_BC_EXTERNAL = 0, 1, 2, 3, 4, 5
SVE_W, SVE_E, SVE_S, SVE_N = 0, 1, 2, 3
SVE_HOST, SVE_DEVICE = 0, 1

#: every symbol include/sve.h declares
EXPORTS = ("sve_config_default", "sve_create", "sve_set_stream", "sve_set_state", "sve_step", "sve_step_dt",
           "sve_get_state", "sve_get_diag", "sve_get_dts", "sve_destroy", "sve_strerror", "sve_last_launch_count",
           "sve_step_async", "sve_sync", "sve_profile", "sve_profile_read", "sve_get_counters", "sve_step_noalloc",
           "sve_batch_create", "sve_batch_set_stream", "sve_batch_set_state", "sve_batch_step",
           "sve_batch_step_async", "sve_batch_get_state", "sve_batch_get_diag", "sve_batch_get_counters",
           "sve_batch_autotune", "sve_batch_set_schedule", "sve_batch_last_launch_count", "sve_batch_destroy",
           "sve_record_forward", "sve_adjoint", "sve_set_block_size", "sve_get_block_size", "sve_advance",
           "sve_get_checkpoint_every", "sve_set_persistent", "sve_get_persistent", "sve_check_sync_timeout",
           "sve_get_safeguards", "sve_block_get_edge", "sve_block_set_ghosts", "sve_block_speeds",
           "sve_block_advance", "sve_batch_autotune_trials", "sve_batch_set_rows", "sve_batch_get_rows",
           "sve_set_adjoint_budget", "sve_get_adjoint_kept_steps", "sve_set_scheme", "sve_get_scheme",
           "sve_set_history", "sve_get_history")


class sve_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("g", ctypes.c_double), ("cfl", ctypes.c_double),
        ("precision", ctypes.c_int), ("bedload", ctypes.c_int),
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


_LIB = None


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libsve.so (built in-tree).  Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libsve.so not found at {path}: build it with paper_1307_0491_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    cfgp = ctypes.POINTER(sve_config)
    sig = {
        "sve_config_default": ([cfgp], ip),
        "sve_create": ([cfgp, ctypes.POINTER(vp)], ip),
        "sve_set_stream": ([vp, vp], ip),
        "sve_set_state": ([vp, vp, vp, vp, vp, ip], ip),
        "sve_step": ([vp, ip, dp], ip),
        "sve_step_dt": ([vp, ip, dp], ip),
        "sve_get_state": ([vp, vp, vp, vp, vp, ip], ip),
        "sve_advance": ([vp, ip, vp, vp, vp, vp, vp, vp, vp, vp, ip, dp], ip),
        "sve_get_diag": ([vp, dp, dp, dp, dp], ip),
        "sve_get_dts": ([vp, dp, ip], ip),
        "sve_destroy": ([vp], None),
        "sve_strerror": ([ip], ctypes.c_char_p),
        "sve_last_launch_count": ([vp], ctypes.c_longlong),
        "sve_step_async": ([vp, ip], ip),
        "sve_sync": ([vp], ip),
        "sve_profile": ([vp, ip], ip),
        "sve_profile_read": ([vp, dp, ctypes.POINTER(ctypes.c_longlong)], ip),
        "sve_get_counters": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_ulonglong)], ip),
        "sve_get_safeguards": ([vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong),
                                ctypes.POINTER(ctypes.c_ulonglong)], ip),
        "sve_step_noalloc": ([cfgp, vp, vp, vp, vp, ip, dp, vp], ip),
        "sve_batch_create": ([cfgp, ip, ctypes.POINTER(vp)], ip),
        "sve_batch_set_stream": ([vp, vp], ip),
        "sve_batch_set_state": ([vp, ip, vp, vp, vp, vp, ip], ip),
        "sve_batch_step": ([vp, ip], ip),
        "sve_batch_step_async": ([vp, ip], ip),
        "sve_batch_get_state": ([vp, ip, vp, vp, vp, vp, ip], ip),
        "sve_batch_get_diag": ([vp, ip, dp, dp, dp, dp], ip),
        "sve_batch_get_counters": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_ulonglong)], ip),
        "sve_batch_autotune": ([vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip)], ip),
        "sve_batch_set_schedule": ([vp, ip, ip], ip),
        "sve_batch_autotune_trials": ([vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip), dp], ip),
        "sve_batch_set_rows": ([vp, ip], ip),
        "sve_batch_get_rows": ([vp], ip),
        "sve_batch_last_launch_count": ([vp], ctypes.c_longlong),
        "sve_batch_destroy": ([vp], None),
        "sve_record_forward": ([vp, ip, ip], ip),
        "sve_get_checkpoint_every": ([vp], ip),
        "sve_set_adjoint_budget": ([vp, ctypes.c_longlong], ip),
        "sve_set_scheme": ([vp, ip], ip),
        "sve_set_history": ([vp, ip], ip),
        "sve_get_history": ([vp, dp, ip], ip),
        "sve_get_scheme": ([vp], ip),
        "sve_get_adjoint_kept_steps": ([vp], ip),
        "sve_set_persistent": ([vp, ip], ip),
        "sve_get_persistent": ([vp], ip),
        "sve_check_sync_timeout": ([vp, ctypes.c_longlong], ip),
        "sve_adjoint": ([vp, vp, vp, vp, vp, ip, vp, vp, vp, vp, dp], ip),
        "sve_set_block_size": ([vp, ip], ip),
        "sve_block_get_edge": ([vp, ip, vp, ip], ip),
        "sve_block_set_ghosts": ([vp, ip, vp, ip], ip),
        "sve_block_speeds": ([vp, dp, dp], ip),
        "sve_block_advance": ([vp, ctypes.c_double, ctypes.c_double], ip),
        "sve_get_block_size": ([vp], ip),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = L
    return L


# ---- the C ABI, same names ---------------------------------------------------

def sve_config_default(cfg: sve_config) -> int:
    return load().sve_config_default(ctypes.byref(cfg))


def sve_create(cfg: sve_config) -> tuple[int, ctypes.c_void_p]:
    h = ctypes.c_void_p()
    rc = load().sve_create(ctypes.byref(cfg), ctypes.byref(h))
    return rc, h


def sve_set_stream(h, stream: int | None) -> int:
    return load().sve_set_stream(h, ctypes.c_void_p(stream or 0))


def sve_set_state(h, depth: int, hu: int, hv: int | None, zb: int, where: int) -> int:
    return load().sve_set_state(h, depth, hu, hv, zb, where)


def sve_step(h, nsteps: int) -> tuple[int, float]:
    t = ctypes.c_double(0.0)
    rc = load().sve_step(h, int(nsteps), ctypes.byref(t))
    return rc, t.value


def sve_step_dt(h, dts) -> int:
    a = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    return load().sve_step_dt(h, int(a.size), a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))


def sve_get_state(h, depth: int, hu: int, hv: int | None, zb: int, where: int) -> int:
    return load().sve_get_state(h, depth, hu, hv, zb, where)


def sve_advance(h, nsteps: int, inp, out, where: int) -> tuple[int, float]:
    """inp, out: four buffer addresses each (h, hu, hv or None, z)."""
    t = ctypes.c_double(0.0)
    rc = load().sve_advance(h, int(nsteps), *inp, *out, where, ctypes.byref(t))
    return rc, t.value


def sve_get_diag(h) -> tuple[int, dict]:
    vals = [ctypes.c_double() for _ in range(4)]
    rc = load().sve_get_diag(h, *[ctypes.byref(v) for v in vals])
    return rc, dict(mass_h=vals[0].value, mass_z=vals[1].value, t=vals[2].value, dt=vals[3].value)


def sve_get_dts(h, n: int) -> tuple[int, np.ndarray]:
    out = np.zeros(max(n, 1))
    rc = load().sve_get_dts(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n))
    return rc, out[: max(rc, 0)]


def sve_destroy(h) -> None:
    load().sve_destroy(h)


def sve_strerror(code: int) -> str:
    return load().sve_strerror(int(code)).decode()


def sve_last_launch_count(h) -> int:
    return int(load().sve_last_launch_count(h))


def sve_set_block_size(h, threads: int) -> int:
    return load().sve_set_block_size(h, int(threads))


def sve_get_block_size(h) -> int:
    return int(load().sve_get_block_size(h))


def sve_step_async(h, nsteps: int) -> int:
    return load().sve_step_async(h, int(nsteps))


def sve_sync(h) -> int:
    return load().sve_sync(h)


def sve_profile(h, on: bool) -> int:
    return load().sve_profile(h, 1 if on else 0)


def sve_profile_read(h) -> tuple[int, list, list]:
    ms = (ctypes.c_double * 2)()
    n = (ctypes.c_longlong * 2)()
    rc = load().sve_profile_read(h, ms, n)
    return rc, list(ms), list(n)


def sve_get_counters(h) -> tuple[int, int, int]:
    steps = ctypes.c_longlong(0)
    its = ctypes.c_ulonglong(0)
    rc = load().sve_get_counters(h, ctypes.byref(steps), ctypes.byref(its))
    return rc, steps.value, its.value


def sve_get_safeguards(h) -> tuple[int, int, int, int]:
    halv = ctypes.c_ulonglong(0)
    raised = ctypes.c_ulonglong(0)
    retries = ctypes.c_ulonglong(0)
    rc = load().sve_get_safeguards(h, ctypes.byref(halv), ctypes.byref(raised), ctypes.byref(retries))
    return rc, halv.value, raised.value, retries.value


def sve_block_get_edge(h, side: int, edge: int, where: int) -> int:
    return load().sve_block_get_edge(h, int(side), edge, int(where))


def sve_block_set_ghosts(h, side: int, ghosts: int, where: int) -> int:
    return load().sve_block_set_ghosts(h, int(side), ghosts, int(where))


def sve_block_speeds(h) -> tuple[int, float, float]:
    sx, sy = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = load().sve_block_speeds(h, ctypes.byref(sx), ctypes.byref(sy))
    return rc, sx.value, sy.value


def sve_block_advance(h, sx: float, sy: float) -> int:
    return load().sve_block_advance(h, float(sx), float(sy))


def sve_step_noalloc(cfg: sve_config, depth: int, hu: int, hv: int | None, zb: int, nsteps: int, t: float,
                     stream: int | None = None) -> tuple[int, float]:
    """Steps on caller-owned device arrays without any device allocation
    (scratch in the library's static device array); returns (code, time)."""
    tt = ctypes.c_double(t)
    rc = load().sve_step_noalloc(ctypes.byref(cfg), depth, hu, hv, zb, int(nsteps), ctypes.byref(tt),
                                 ctypes.c_void_p(stream or 0))
    return rc, tt.value


def sve_batch_create(cfgs) -> tuple[int, ctypes.c_void_p]:
    arr = (sve_config * len(cfgs))(*cfgs)
    b = ctypes.c_void_p()
    rc = load().sve_batch_create(arr, len(cfgs), ctypes.byref(b))
    return rc, b


def sve_batch_set_state(b, run: int, depth: int, hu: int, hv: int | None, zb: int, where: int) -> int:
    return load().sve_batch_set_state(b, int(run), depth, hu, hv, zb, where)


def sve_batch_step(b, nsteps: int) -> int:
    return load().sve_batch_step(b, int(nsteps))


def sve_batch_step_async(b, nsteps: int) -> int:
    return load().sve_batch_step_async(b, int(nsteps))


def sve_batch_get_state(b, run: int, depth: int, hu: int, hv: int | None, zb: int, where: int) -> int:
    return load().sve_batch_get_state(b, int(run), depth, hu, hv, zb, where)


def sve_batch_get_diag(b, run: int) -> tuple[int, dict]:
    vals = [ctypes.c_double() for _ in range(4)]
    rc = load().sve_batch_get_diag(b, int(run), *[ctypes.byref(v) for v in vals])
    return rc, dict(mass_h=vals[0].value, mass_z=vals[1].value, t=vals[2].value, dt=vals[3].value)


def sve_batch_get_counters(b) -> tuple[int, int, int]:
    steps = ctypes.c_longlong(0)
    its = ctypes.c_ulonglong(0)
    rc = load().sve_batch_get_counters(b, ctypes.byref(steps), ctypes.byref(its))
    return rc, steps.value, its.value


def sve_batch_autotune(b, trial_steps: int) -> tuple[int, int, int]:
    tile, sched = ctypes.c_int(0), ctypes.c_int(0)
    rc = load().sve_batch_autotune(b, int(trial_steps), ctypes.byref(tile), ctypes.byref(sched))
    return rc, tile.value, sched.value


def sve_batch_set_schedule(b, tile: int, schedule: int) -> int:
    return load().sve_batch_set_schedule(b, int(tile), int(schedule))


def sve_batch_set_stream(b, stream: int | None) -> int:
    return load().sve_batch_set_stream(b, ctypes.c_void_p(stream or 0))


def sve_batch_last_launch_count(b) -> int:
    return int(load().sve_batch_last_launch_count(b))


def sve_batch_destroy(b) -> None:
    load().sve_batch_destroy(b)


def sve_record_forward(h, nsteps: int, checkpoint_every: int = 0) -> int:
    return load().sve_record_forward(h, int(nsteps), int(checkpoint_every))


def sve_adjoint(h, lam: tuple, where: int, grads: tuple) -> tuple[int, list]:
    """lam = (lam_h, lam_hu, lam_hv, lam_z) pointers (or None); grads = four
    output pointers (or None).  Returns (code, [dL/dA_g, dL/dm_g, dL/dK])."""
    g = (ctypes.c_double * 3)()
    rc = load().sve_adjoint(h, *lam, where, *grads, g)
    return rc, list(g)


# ---- convenience wrapper ---------------------------------------------------

class SveError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {sve_strerror(code)} ({code})")
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise SveError(rc, where)
    return rc


_BEDLOAD = {"grass": SVE_GRASS, "mpm": SVE_MPM, "flvb": SVE_FLVB, "nielsen": SVE_NIELSEN,
            "ribberink": SVE_RIBBERINK, "camenen": SVE_CAMENEN}
_FRICTION = {"none": SVE_FRIC_NONE, "darcy": SVE_FRIC_DARCY, "strickler": SVE_FRIC_STRICKLER}
_BC = {"periodic": SVE_BC_PERIODIC, "free": SVE_BC_FREE, "inflow_q": SVE_BC_INFLOW_Q,
       "inflow_qh": SVE_BC_INFLOW_QH, "wall": SVE_BC_WALL, "external": SVE_BC_EXTERNAL}


def config_from_params(p: dict, precision: str = "fp64") -> sve_config:
    """sve_config from a workload parameter dict (string-valued enums)."""
    c = sve_config()
    _check(sve_config_default(c), "sve_config_default")
    for name, _ in sve_config._fields_:
        if name in ("bc", "precision", "bedload", "friction"):
            continue
        if name in p:
            setattr(c, name, p[name])
    c.precision = SVE_FP64 if precision == "fp64" else SVE_FP32
    c.bedload = _BEDLOAD[p["bedload"]] if isinstance(p.get("bedload"), str) else int(p.get("bedload", 0))
    c.friction = _FRICTION[p["friction"]] if isinstance(p.get("friction"), str) else int(p.get("friction", 0))
    bc = p.get("bc", ("periodic", "periodic", "free", "free"))
    c.bc = (ctypes.c_int * 4)(*[_BC[b] if isinstance(b, str) else int(b) for b in bc])
    return c


class Solver:
    """One SVE simulation on the current CUDA device (owns a libsve handle)."""

    def __init__(self, params: dict, precision: str = "fp64", stream: int | None = None):
        self.params = dict(params)
        self.precision = precision
        self.dtype = np.float64 if precision == "fp64" else np.float32
        self.dim = int(params["dim"])
        self.nx, self.ny = int(params["nx"]), int(params["ny"]) if int(params["dim"]) == 2 else 1
        self.cfg = config_from_params(params, precision)
        rc, self.h = sve_create(self.cfg)
        _check(rc, "sve_create")
        if stream is not None:
            _check(sve_set_stream(self.h, stream), "sve_set_stream")

    def close(self):
        if getattr(self, "h", None):
            sve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self):
        return (self.ny, self.nx) if self.dim == 2 else (self.nx,)

    def set_state(self, h, hu, hv, z):
        """Host arrays (numpy) or CUDA tensors (torch); copied in."""
        if hasattr(h, "is_cuda") and h.is_cuda:
            ts = [x.contiguous() for x in (h, hu, z)]
            hvp = hv.contiguous().data_ptr() if (self.dim == 2 and hv is not None) else None
            self._keep = ts
            return _check(sve_set_state(self.h, ts[0].data_ptr(), ts[1].data_ptr(), hvp, ts[2].data_ptr(),
                                        SVE_DEVICE), "sve_set_state")
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=self.dtype).reshape(self._shape())) for x in (h, hu, z)]
        hva = (np.ascontiguousarray(np.asarray(hv, dtype=self.dtype).reshape(self._shape()))
               if self.dim == 2 else None)
        return _check(sve_set_state(self.h, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                    hva.ctypes.data if hva is not None else None, arrs[2].ctypes.data, SVE_HOST),
                      "sve_set_state")

    def step(self, nsteps: int) -> float:
        rc, t = sve_step(self.h, nsteps)
        _check(rc, "sve_step")
        return t

    def step_dt(self, dts) -> None:
        _check(sve_step_dt(self.h, dts), "sve_step_dt")

    def get_state(self) -> dict:
        shp = self._shape()
        out = {k: np.empty(shp, dtype=self.dtype) for k in ("h", "hu", "z")}
        out["hv"] = np.empty(shp, dtype=self.dtype) if self.dim == 2 else None
        _check(sve_get_state(self.h, out["h"].ctypes.data, out["hu"].ctypes.data,
                             out["hv"].ctypes.data if out["hv"] is not None else None, out["z"].ctypes.data,
                             SVE_HOST), "sve_get_state")
        return out

    def advance(self, nsteps: int, inp: dict, out: dict) -> float:
        """sve_advance from the arrays of ``inp`` to those of ``out`` (keys
        h, hu, hv, z; numpy arrays -- page-locked if they come from a pinned
        torch tensor's ``.numpy()`` -- or CUDA tensors, all of one kind, of
        the state dtype, contiguous); returns the simulated time."""
        def addr(a):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                return a.data_ptr()
            if not (a.flags["C_CONTIGUOUS"] and a.dtype == self.dtype):
                raise ValueError("sve_advance: contiguous arrays of the state dtype required")
            return a.ctypes.data
        keys = ("h", "hu", "hv", "z")
        on_dev = [bool(getattr(x[k], "is_cuda", False)) for x in (inp, out) for k in keys if x.get(k) is not None]
        if any(on_dev) and not all(on_dev):
            raise ValueError("sve_advance: all buffers on the host or all on the device")
        where = SVE_DEVICE if on_dev and on_dev[0] else SVE_HOST
        rc, t = sve_advance(self.h, nsteps, [addr(inp.get(k)) for k in keys], [addr(out.get(k)) for k in keys],
                            where)
        _check(rc, "sve_advance")
        return t

    def get_state_device(self, h, hu, hv, z) -> None:
        """Copy the state into CUDA tensors (contiguous, state dtype)."""
        _check(sve_get_state(self.h, h.data_ptr(), hu.data_ptr(), hv.data_ptr() if hv is not None else None,
                             z.data_ptr(), SVE_DEVICE), "sve_get_state")

    def diag(self) -> dict:
        rc, d = sve_get_diag(self.h)
        _check(rc, "sve_get_diag")
        return d

    def dts(self, n: int) -> np.ndarray:
        rc, d = sve_get_dts(self.h, n)
        _check(rc, "sve_get_dts")
        return d

    def launches(self) -> int:
        return sve_last_launch_count(self.h)

    def step_async(self, nsteps: int) -> None:
        _check(sve_step_async(self.h, nsteps), "sve_step_async")

    def set_persistent(self, on: int) -> None:
        """1: persistent cooperative launches when eligible, 0: the two
        kernels from CUDA graphs (the default) -- sve_set_persistent."""
        _check(load().sve_set_persistent(self.h, int(on)), "sve_set_persistent")

    def persistent(self) -> bool:
        return load().sve_get_persistent(self.h) == 1

    def set_block_size(self, threads: int) -> None:
        """Threads per block of the two-kernel step: 0 (automatic), 32, 128 or 256."""
        _check(sve_set_block_size(self.h, threads), "sve_set_block_size")

    @property
    def block_size(self) -> int:
        return sve_get_block_size(self.h)

    def sync(self) -> None:
        _check(sve_sync(self.h), "sve_sync")

    def profile(self, on: bool) -> None:
        _check(sve_profile(self.h, on), "sve_profile")

    def profile_read(self) -> dict:
        rc, ms, n = sve_profile_read(self.h)
        _check(rc, "sve_profile_read")
        return dict(iface_ms=ms[0], cell_ms=ms[1], iface_launches=n[0], cell_launches=n[1])

    def counters(self) -> dict:
        rc, steps, its = sve_get_counters(self.h)
        _check(rc, "sve_get_counters")
        return dict(steps=steps, newton_iters=its)

    # -- one block of a decomposed grid (sides marked "external") ----------
    def edge(self, side: int) -> np.ndarray:
        """The interior cells along a side: (4, n) array (h, hu, hv, z)."""
        n = self.ny if side in (SVE_W, SVE_E) else self.nx
        out = np.empty((4, n), dtype=self.dtype)
        _check(sve_block_get_edge(self.h, side, out.ctypes.data, SVE_HOST), "sve_block_get_edge")
        return out

    def set_ghosts(self, side: int, ghosts) -> None:
        """The ghost ring of an external side from a (4, n) array."""
        g = np.ascontiguousarray(np.asarray(ghosts, dtype=self.dtype))
        _check(sve_block_set_ghosts(self.h, side, g.ctypes.data, SVE_HOST), "sve_block_set_ghosts")

    def block_speeds(self) -> tuple[float, float]:
        rc, sx, sy = sve_block_speeds(self.h)
        _check(rc, "sve_block_speeds")
        return sx, sy

    def block_advance(self, sx: float, sy: float) -> None:
        _check(sve_block_advance(self.h, sx, sy), "sve_block_advance")

    def safeguards(self) -> dict:
        rc, halv, raised, retries = sve_get_safeguards(self.h)
        _check(rc, "sve_get_safeguards")
        return dict(halvings=halv, raised=raised, retries=retries)

    def checkpoint_every(self) -> int:
        """The recording's checkpoint interval (nsteps: every step kept)."""
        n = load().sve_get_checkpoint_every(self.h)
        _check(min(n, 0), "sve_get_checkpoint_every")
        return n

    def set_history(self, capacity: int) -> None:
        """Keep a record (t, dt, mass_h, mass_z, Sx, Sy) after every later
        step in a device ring of `capacity` records (0: off) -- sve_set_history."""
        _check(load().sve_set_history(self.h, int(capacity)), "sve_set_history")

    def history(self, n: int) -> np.ndarray:
        """The last records, oldest first: an (m, 6) array (t, dt, mass_h,
        mass_z, Sx, Sy), m <= n."""
        out = np.zeros((max(n, 1), 6))
        m = load().sve_get_history(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(n))
        _check(min(m, 0), "sve_get_history")
        return out[:m]

    def set_scheme(self, scheme: str) -> None:
        """"coupled" (the paper's step, the default) or "split" (the
        splitting scheme it is contrasted with: a shallow-water step, then
        an upwind Exner update of the bed) -- sve_set_scheme."""
        code = {"coupled": SVE_SCHEME_COUPLED, "split": SVE_SCHEME_SPLIT}[scheme]
        _check(load().sve_set_scheme(self.h, code), "sve_set_scheme")

    @property
    def scheme(self) -> str:
        return "split" if load().sve_get_scheme(self.h) == SVE_SCHEME_SPLIT else "coupled"

    def adjoint_kept_steps(self) -> int:
        """How many recorded steps' forward data the recording kept."""
        n = load().sve_get_adjoint_kept_steps(self.h)
        _check(min(n, 0), "sve_get_adjoint_kept_steps")
        return n

    def set_adjoint_budget(self, nbytes: int) -> None:
        """Bytes of forward data the next automatic recordings may keep (-1:
        half of the free device memory)."""
        _check(load().sve_set_adjoint_budget(self.h, int(nbytes)), "sve_set_adjoint_budget")

    def record_forward(self, nsteps: int, checkpoint_every: int = 0) -> None:
        _check(sve_record_forward(self.h, nsteps, checkpoint_every), "sve_record_forward")

    def adjoint(self, lam_h=None, lam_hu=None, lam_hv=None, lam_z=None) -> tuple[dict, list]:
        """Host cotangents of the final state -> (dL/dU^0 as numpy arrays,
        [dL/dA_g, dL/dm_g, dL/dK])."""
        shp = self._shape()
        lam = []
        keep = []
        for x in (lam_h, lam_hu, lam_hv, lam_z):
            if x is None:
                lam.append(None)
            else:
                a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(shp))
                keep.append(a)
                lam.append(a.ctypes.data)
        out = {k: np.zeros(shp) for k in ("h", "hu", "hv", "z")}
        ptrs = tuple(out[k].ctypes.data if (k != "hv" or self.dim == 2) else None for k in ("h", "hu", "hv", "z"))
        rc, gp = sve_adjoint(self.h, tuple(lam), SVE_HOST, ptrs)
        _check(rc, "sve_adjoint")
        if self.dim == 1:
            out["hv"] = None
        return out, gp


class Batch:
    """An ensemble of independent runs stepped together (sve_batch_*)."""

    def __init__(self, params_list, precision: str = "fp64", stream: int | None = None):
        self.params = [dict(p) for p in params_list]
        self.precision = precision
        self.dtype = np.float64 if precision == "fp64" else np.float32
        cfgs = [config_from_params(p, precision) for p in self.params]
        rc, self.h = sve_batch_create(cfgs)
        _check(rc, "sve_batch_create")
        if stream is not None:
            _check(sve_batch_set_stream(self.h, stream), "sve_batch_set_stream")

    def close(self):
        if getattr(self, "h", None):
            sve_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, r):
        p = self.params[r]
        return (p["ny"], p["nx"]) if p["dim"] == 2 else (p["nx"],)

    def set_state(self, r: int, h, hu, hv, z):
        arrs = [np.ascontiguousarray(np.asarray(x, dtype=self.dtype).reshape(self._shape(r))) for x in (h, hu, z)]
        hva = (np.ascontiguousarray(np.asarray(hv, dtype=self.dtype).reshape(self._shape(r)))
               if self.params[r]["dim"] == 2 else None)
        _check(sve_batch_set_state(self.h, r, arrs[0].ctypes.data, arrs[1].ctypes.data,
                                   hva.ctypes.data if hva is not None else None, arrs[2].ctypes.data, SVE_HOST),
               "sve_batch_set_state")

    def step(self, nsteps: int) -> None:
        _check(sve_batch_step(self.h, nsteps), "sve_batch_step")

    def step_async(self, nsteps: int) -> None:
        _check(sve_batch_step_async(self.h, nsteps), "sve_batch_step_async")

    def get_state(self, r: int) -> dict:
        shp = self._shape(r)
        out = {k: np.empty(shp, dtype=self.dtype) for k in ("h", "hu", "z")}
        out["hv"] = np.empty(shp, dtype=self.dtype) if self.params[r]["dim"] == 2 else None
        _check(sve_batch_get_state(self.h, r, out["h"].ctypes.data, out["hu"].ctypes.data,
                                   out["hv"].ctypes.data if out["hv"] is not None else None, out["z"].ctypes.data,
                                   SVE_HOST), "sve_batch_get_state")
        return out

    def diag(self, r: int) -> dict:
        rc, d = sve_batch_get_diag(self.h, r)
        _check(rc, "sve_batch_get_diag")
        return d

    def counters(self) -> dict:
        rc, steps, its = sve_batch_get_counters(self.h)
        _check(rc, "sve_batch_get_counters")
        return dict(steps=steps, newton_iters=its)

    def autotune(self, trial_steps: int = 3) -> tuple[int, int]:
        rc, tile, sched = sve_batch_autotune(self.h, trial_steps)
        _check(rc, "sve_batch_autotune")
        return tile, sched

    def set_schedule(self, tile: int, schedule: int) -> None:
        _check(sve_batch_set_schedule(self.h, tile, schedule), "sve_batch_set_schedule")

    def trials(self) -> list[dict]:
        """The last autotune's candidates and their mean trial-step times."""
        L = load()
        n = L.sve_batch_autotune_trials(self.h, 0, None, None, None, None)
        _check(min(n, 0), "sve_batch_autotune_trials")
        t, s, r = (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))()
        ms = (ctypes.c_double * max(n, 1))()
        L.sve_batch_autotune_trials(self.h, n, t, s, r, ms)
        return [dict(tile=t[k], schedule=s[k], rows=r[k], ms_per_step=ms[k]) for k in range(n)]

    def set_rows(self, rows: int) -> None:
        _check(load().sve_batch_set_rows(self.h, int(rows)), "sve_batch_set_rows")

    @property
    def rows(self) -> int:
        return load().sve_batch_get_rows(self.h)
