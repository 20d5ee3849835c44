#!/usr/bin/env python
"""Benchmark of the Saint-Venant--Exner relaxation step on GB300.

Workload: the 2D dune channel, FP64 (1024 x 512 cells over 1000 x 500 m,
Gaussian dune, Grass m_g = 3, A_g = 1e-3, Strickler K = 40, inflow / free
boundaries).  One "step" = one time step of the whole hot path: interface
Riemann solves + CFL reduction (interface kernel) and cell update +
friction + projection + ghosts + mass sums (cell kernel).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  N > 1 (torchrun): every rank runs its own
replica of the workload (independent runs, no data-path collective: weak
scaling); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import datetime
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D cell-updates/s"
UNIT = "cell-updates/s"
BYTES_PER_CELL_FP64 = 64           # read h, hu, hv, zb once + write once (FP64)
# algorithmic FP64 operations of one interface solve (+, -, *, /, sqrt
# counted as one each; comparisons not counted), from the operation list of
# the solver: celerities and constants, one F/F' evaluation, one Newton
# update, intermediate states and fluctuations
FLOP_SETUP, FLOP_EVAL, FLOP_UPDATE, FLOP_FINAL = 30, 76, 4, 75
FP64_PEAK_FLOPS = 152 * 2 * 2 * 2070e6   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
FP32_PEAK_FLOPS = 152 * 128 * 2 * 2070e6  # 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one interface-kernel launch on this workload,
# from the ncu capture summarised in profiles/interface_kernel_dune2d_fp64_1024x512.md,
# valid only for the kernel source it was taken with (sha256 prefix)
IFACE_TRAFFIC = {"sha256": "b0de5f66329ab712", "bytes": 94_304_256}


def workload_desc(nx, ny, workload="dune2d", precision="fp64"):
    if workload == "antidune2d":
        return (f"2D antidune {precision.upper()} {nx}x{ny} (24x12 m, bed N(0, 1 cm), h=0.5 m, Fr~U[1.2,1.5], "
                f"MPM + Darcy f=0.02, supercritical inflow / free)")
    return (f"2D dune {precision.upper()} {nx}x{ny} (1000x500 m, Gaussian dune, Grass m_g=3 A_g=1e-3, "
            f"Strickler K=40, inflow q=0.5 / free outflow)")


def bench_config(args, nx, ny):
    """The `config` of the JSON line, the same for both arms: the workload,
    its grid and precision, the window of the run the timed steps cover
    (after --spinup untimed steps and the warm-up steps) and how L2 is
    kept out of the timing."""
    return {"workload": workload_desc(nx, ny, args.workload, args.precision), "nx": nx, "ny": ny,
            "precision": args.precision,
            "timed_steps_of_run": f"{args.spinup + args.warmup}..{args.spinup + args.warmup + args.steps - 1}",
            "per_rank": "independent replica (seed = rank)",
            "l2": f"GPU arm: {L2_FLUSH_BYTES >> 20} MiB written between timed steps, outside the events "
                  f"(L2 flush); CPU arm: no flush"}


def make_workload(args, W, seed=0):
    """The timed workload: the 2D dune (default, FP64) or the antidune (its
    FP32 and FP64 forms); --nx/--ny shrink it (profiling captures)."""
    if args.workload == "antidune2d":
        kw = {}
        if args.nx:
            kw.update(nx=args.nx, ny=args.ny or args.nx // 2)
        return W.antidune2d(seed=seed, **kw)
    kw = {}
    if args.nx:
        kw.update(nx=args.nx, ny=args.ny or args.nx // 2)
    return W.dune2d(seed=seed, **kw)


def iface_traffic():
    """Measured traffic per launch, or None if the kernel changed since."""
    import hashlib

    src = os.path.join(ROOT, "paper_1307_0491_gb300", "csrc", "sve_device.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return IFACE_TRAFFIC["bytes"] if sha == IFACE_TRAFFIC["sha256"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms; only the
    samples stamped inside the marked region count."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self, wait_s: float = 5.0):
        """Start sampling and wait for the first sample (so that the region
        marked next is covered)."""
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        end = time.time() + wait_s
        while time.time() < end and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = datetime.datetime.now()

    def mark_end(self):
        self.t1 = datetime.datetime.now()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows, unstamped = [], []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                unstamped.append(parts[1:])
                continue
            rows.append((ts, parts[1:]))
        os.remove(self.path)
        if not rows and unstamped:  # timestamps in an unexpected format: every sample
            rows = [(None, r) for r in unstamped]
            self.t0 = None
        inside = [r for ts, r in rows if self.t0 is not None and self.t0 <= ts <= self.t1]
        use = inside
        if not use and rows:
            if self.t0 is None:
                use = [r for _, r in rows]
            else:  # region shorter than a sample interval: the nearest sample
                mid = self.t0 + (self.t1 - self.t0) / 2
                use = [min(rows, key=lambda x: abs((x[0] - mid).total_seconds()))[1]]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in use if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in use if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(use), "samples_in_region": len(inside),
                "interval_ms": 50}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _oracle_stepper(o, P, st, threads: int):
    """A callable advancing the oracle state by n steps: the whole-grid
    stepper on one thread, or the row-banded oracle on ``threads`` threads
    (2D; bit-identical results)."""
    from oracle.banded import BandedRun

    if threads > 1 and P.dim == 2:
        run = BandedRun(o, P, *st, nbands=threads, threads=threads)
        return run.step, run.close
    cur = {"st": st}

    def step(n):
        r = o.run(P, n, *cur["st"])
        cur["st"] = (r["h"], r["hu"], r["hv"], r["z"])

    return step, (lambda: None)


def cpu_oracle_rate(w, threads: int, budget_s: float = 10.0, max_steps: int = 5000, state=None):
    """The FP64 oracle on the host, as it stands, on the full grid of the
    workload for as many steps as fit in about budget_s (at least 1), on
    ``threads`` threads (row bands of the oracle's block API when > 1),
    from `state` (h, hu, hv, z; default: the workload's initial state)."""
    import oracle

    o = oracle.get()
    P = oracle.Params.from_workload(w["params"])
    cells = w["params"]["nx"] * w["params"]["ny"]
    st = state if state is not None else (w["h"], w["hu"], w["hv"], w["z"])
    step, close = _oracle_stepper(o, P, st, threads)
    try:
        t0 = time.perf_counter()
        step(1)
        first = time.perf_counter() - t0
        more = int(max(0, min(max_steps - 1, math.floor(budget_s / max(first, 1e-9)) - 1)))
        if more > 0:
            t2 = time.perf_counter()
            step(more)
            steps, secs = more, time.perf_counter() - t2
        else:
            steps, secs = 1, first
    finally:
        close()
    return cells * steps / secs, steps, secs


def oracle_spinup(w, threads: int, nsteps: int):
    """The workload's state after nsteps oracle steps (untimed; row bands on
    `threads` threads, bit-identical to the single-threaded oracle)."""
    import oracle
    from oracle.banded import BandedRun

    o = oracle.get()
    P = oracle.Params.from_workload(w["params"])
    st = (w["h"], w["hu"], w["hv"], w["z"])
    if nsteps <= 0:
        return st
    if threads > 1 and P.dim == 2:
        run = BandedRun(o, P, *st, nbands=threads, threads=threads)
        try:
            run.step(nsteps)
            f = run.state()
        finally:
            run.close()
        return (f["h"], f["hu"], f["hv"], f["z"])
    r = o.run(P, nsteps, *st)
    return (r["h"], r["hu"], r["hv"], r["z"])


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle timed on all host cores (row bands
    of the oracle's block API on threads), one full-grid step per step, over
    the same window of the run as the GPU arm (--spinup untimed steps, the
    warm-up steps, then the timed ones)."""
    if rank != 0:
        return 0
    import oracle
    from oracle.banded import host_threads
    from paper_1307_0491_gb300 import workloads as W

    w = make_workload(args, W)
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    o = oracle.get()
    P = oracle.Params.from_workload(w["params"])
    st = (w["h"], w["hu"], w["hv"], w["z"])
    threads = host_threads()
    # one full-grid step sets the size of the sample: if all steps on the
    # full grid would take more than ~2 minutes, every step runs on the first
    # ny' rows of the workload (same physics and boundary types)
    step, close = _oracle_stepper(o, P, st, threads)
    t0 = time.perf_counter()
    step(1)
    t_full = time.perf_counter() - t0
    close()
    budget = 150.0
    ny_full = ny
    sample = f"full {nx}x{ny} grid"
    total = args.spinup + args.steps + args.warmup
    if total * t_full > budget and w["params"]["dim"] == 2:
        nys = max(8 * threads, int(ny * budget / (total * t_full)))
        nys = min(nys, ny)
        p2 = dict(w["params"], ny=nys, ly=w["params"]["ly"] * nys / ny)
        w = dict(w, params=p2, h=w["h"][:nys], hu=w["hu"][:nys], hv=w["hv"][:nys], z=w["z"][:nys])
        ny = nys
        P = oracle.Params.from_workload(p2)
        st = (w["h"], w["hu"], w["hv"], w["z"])
        sample = f"rows 0..{nys - 1} of the {nx}x{ny_full} grid"
    step, close = _oracle_stepper(o, P, st, threads)
    try:
        if args.spinup > 0:
            step(args.spinup)
        step(args.warmup)
        t0 = time.perf_counter()
        step(args.steps)
        secs = time.perf_counter() - t0
    finally:
        close()
    value = nx * ny * args.steps / secs
    how = (f"C oracle (-O2, no FMA contraction) on {threads} threads, row bands of its block API"
           if threads > 1 and P.dim == 2 else "single-threaded C oracle (-O2, no FMA contraction)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, nx, ny_full),
        "cpu_baseline": {"kind": "oracle", "cores": threads if P.dim == 2 else 1, "value": value, "unit": UNIT,
                         "sample": f"{sample}, {args.steps} steps after {args.spinup} spin-up and {args.warmup} "
                                   f"warm-up steps, {how}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, sve, W, torch, precision: str, plain_value: float):
    """The batched ensemble: 256 independent 2D dune runs of uneven sizes and
    parameters stepped together; cell-updates/s over all runs, compared with
    the plain single-run step of the same precision."""
    runs = W.ensemble(nruns=args.batch_runs, seed=0)
    cells = sum(r["params"]["nx"] * r["params"]["ny"] for r in runs)
    b = sve.Batch([r["params"] for r in runs], precision, stream=torch.cuda.current_stream().cuda_stream)
    for i, r in enumerate(runs):
        b.set_state(i, r["h"], r["hu"], r["hv"], r["z"])
    tile, sched = b.autotune(10)
    trials = b.trials()
    rows = b.rows
    b.step(args.batch_spinup)
    b.step(3)
    c0 = b.counters()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step_async(args.batch_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    c1 = b.counters()
    b.close()
    value = cells * args.batch_steps / (ms * 1e-3)
    return {"workload": f"{args.batch_runs} independent 2D dune runs, Nx~U{{128..1024}}, Ny~U{{64..512}}, "
                        f"A_g log-U[1e-4,1e-2], m_g in {{1,2,3,4}}, amplitude U[0.2,1] (seed 0)",
            "precision": precision, "runs": args.batch_runs, "cells_per_step": cells, "value": value, "unit": UNIT,
            "ms_per_step": ms / args.batch_steps, "steps": args.batch_steps,
            "timed_steps_of_run": f"{args.batch_spinup + 3}..{args.batch_spinup + 2 + args.batch_steps}",
            "launches_per_step": 2, "tile": tile, "schedule": ["run-major", "round-robin"][sched],
            "rows_per_strip_run": rows or None,
            "solve_pass": "marching strips (fused FP32 step)" if rows else "interface tiles (two-kernel step)",
            "autotune": {"trial_steps": 10, "candidates": trials},
            "newton_updates": c1["newton_iters"] - c0["newton_iters"],
            "vs_plain": value / plain_value if plain_value else None,
            "l2": "working set larger than L2 (no flush)"}


def run_adjoint(args, sve, W, torch):
    """Gradient of ||z_b(T) - z_target||^2 with respect to A_g, m_g, K and the
    initial bed on the adjoint config (2048 x 1024, periodic), over a bounded
    number of steps: forward record + reverse sweep, against the plain
    forward step on the same grid."""
    w = W.adjoint_dune()
    tgt = W.adjoint_dune(A_g=1.1e-3, m_g=3.1, K_st=36.0, shift=5.0)
    p = w["params"]
    cells = p["nx"] * p["ny"]
    n = args.adjoint_steps
    # target bed: a forward run of the perturbed setup
    st = sve.Solver(tgt["params"], "fp64")
    st.set_state(tgt["h"], tgt["hu"], tgt["hv"], tgt["z"])
    st.step(n)
    z_target = st.get_state()["z"]
    st.close()
    s = sve.Solver(p, "fp64")
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(n)                                   # plain forward on the same grid
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    def gradient(every):
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.record_forward(n, every)
        fin = s.get_state()
        t1 = time.perf_counter()
        kept = s.adjoint_kept_steps()
        grads, gp = s.adjoint(lam_z=2.0 * (fin["z"] - z_target))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return grads, gp, t0, t1, t2, (s.checkpoint_every(), kept), fin

    # automatic checkpointing (every step kept when it fits in device memory,
    # else checkpoints every ceil(sqrt(N)) steps with the segments
    # recomputed); the latter also timed on its own when the first kept all
    sq = int(math.ceil(math.sqrt(n)))
    grads, gp, t0, t1, t2, (every, kept), fin = gradient(0)
    if every == n:
        _, _, c0, _, c2, _, _ = gradient(sq)
    else:
        c0, c2 = t0, t2
    # the same recording, reversed for a cotangent that is nonzero in every
    # cell (L = ||z(T)||^2): the misfit above is zero where both runs stayed
    # uniform, and interfaces with zero cotangents on both sides are skipped
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    s.adjoint(lam_z=2.0 * fin["z"])
    torch.cuda.synchronize()
    dense_rev = time.perf_counter() - t3
    s.close()
    plain = cells * n / t_plain
    grad_rate = cells * n / (t2 - t0)
    return {"workload": f"adjoint config {p['nx']}x{p['ny']} periodic, dune physics in 2D, Grass A_g=1e-3 m_g=3, "
                        f"Strickler K=40; misfit to a (1.1 A_g, m_g=3.1, K=36, +5 m) run",
            "steps": n, "checkpoint_every": every,
            "storage": "every step's state kept in device memory" if every == n else
            f"checkpoints every {every} steps; the last {kept} steps' forward data kept in device memory "
            "(half of the free memory), the earlier segments recomputed",
            "kept_steps": kept,
            "checkpointed_value": cells * n / (c2 - c0), "checkpointed_every": sq,
            "value": grad_rate, "unit": "cell-updates/s (forward record + reverse sweep)",
            "plain_forward_value": plain, "vs_plain": grad_rate / plain,
            "forward_record_s": t1 - t0, "reverse_s": t2 - t1,
            "dense_cotangent": {"reverse_s": dense_rev, "value": cells * n / (t1 - t0 + dense_rev),
                                "vs_plain": cells * n / (t1 - t0 + dense_rev) / plain,
                                "functional": "||z_b(T)||^2 (cotangent nonzero in every cell)"},
            "grad_params": {"A_g": gp[0], "m_g": gp[1], "K": gp[2]},
            "grad_z0_max_abs": float(np.max(np.abs(grads["z"]))), "dtype": "f64",
            "time": "wall clock around the C-ABI calls (host-synchronous)"}


def run_splitting(args, sve, W, torch):
    """The splitting scheme Sec. 2 contrasts with the coupled method (a
    shallow-water step, then an upwind Exner update of the bed;
    sve_set_scheme) against the coupled step, on the paper's 1D dune (1000 m,
    h = 10 - z_b, q0 = 10, Grass A_g = 1, m_g = 3) at J = 2000 for 2000 CFL
    steps: steps per second of each (wall clock around one host-synchronous
    sve_step call) and the bed it leaves -- total variation, local extrema,
    crest and trough."""
    w = W.paper_dune1d(nx=2000, A_g=1.0)
    n = 2000

    def bed(z):
        dz = np.diff(np.asarray(z, dtype=np.float64))
        return {"total_variation": float(np.sum(np.abs(dz))),
                "local_extrema": int(np.sum(np.sign(dz[1:]) * np.sign(dz[:-1]) < 0)),
                "z_max": float(np.max(z)), "z_min": float(np.min(z))}

    out = {"workload": "1D dune (Sec. 5.1 setting: 1000 m, h = 10 - z_b, q0 = 10, Grass A_g = 1, m_g = 3), "
                       "2000 cells, 2000 CFL steps", "steps": n, "initial_bed": bed(w["z"])}
    for scheme in ("coupled", "split"):
        s = sve.Solver(w["params"], "fp64")
        s.set_scheme(scheme)
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        s.step(16)  # graphs captured
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = s.step(n)
        dt = time.perf_counter() - t0
        out[scheme] = {"steps_per_s": n / dt, "t_end": t, "bed": bed(s.get_state()["z"])}
        s.close()
    out["time"] = "wall clock around one host-synchronous sve_step call of all steps"
    return out


def run_small1d(args, sve, W, torch):
    """Small 1D grids, where a step is a few microseconds of work and its FP64
    work has to be spread over many SMs: the 1D dune (1000 cells, periodic,
    5000 CFL steps) and the 1D antidune of Sec. 5.2 at J = 2400 (5 cm bump):
    the two-kernel step from CUDA graphs of 16 steps with one-warp blocks
    (the automatic choice here) and with 128-thread blocks, and the opt-in
    persistent cooperative step (up to 4096 steps per launch)."""
    out = []
    for name, w, n in (("1D dune 1000 cells periodic, Grass A_g=1e-3 m_g=3, 5000 CFL steps", W.dune1d(), 5000),
                       ("1D antidune (Sec. 5.2) 2400 cells, 5 cm bump, supercritical inflow, 5000 CFL steps",
                        W.paper_antidune1d(nx=2400, bump=0.05), 5000)):
        row = {"workload": name, "steps": n}
        for key, bs, pers in (("persistent", 32, 1), ("block32", 32, 0), ("block128", 128, 0)):
            s = sve.Solver(w["params"], "fp64")
            s.set_block_size(bs)
            s.set_persistent(pers)
            used = s.persistent()
            s.set_state(w["h"], w["hu"], w["hv"], w["z"])
            s.step(200)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.step(n)
            t1 = time.perf_counter()
            launches = s.launches()
            s.close()
            row[key] = {"steps_per_s": n / (t1 - t0), "cell_updates_per_s": n * w["params"]["nx"] / (t1 - t0),
                        "launches": launches, "persistent": used}
        row["persistent_vs_graphs"] = row["persistent"]["steps_per_s"] / row["block32"]["steps_per_s"]
        row["narrow_vs_wide"] = row["block32"]["steps_per_s"] / row["block128"]["steps_per_s"]
        row["time"] = "wall clock around one host-synchronous sve_step call of all steps"
        out.append(row)
    return out


def run_closures(args, sve, W, torch):
    """Each Shields-parameter transport law of Sec. 2 on the antidune physics
    (2048 x 1024 crop of the antidune config: supercritical inflow, random
    bed, Darcy-Weisbach tau*, tau* ~ 1), FP64, 50 timed CFL steps after 20."""
    out = []
    for law in ("mpm", "flvb", "nielsen", "ribberink", "camenen"):
        w = W.antidune2d(nx=2048, ny=1024, seed=0)
        w["params"].update(bedload=law)
        s = sve.Solver(w["params"], "fp64")
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        s.step(20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(50)
        t1 = time.perf_counter()
        its = s.counters()["newton_iters"]
        s.close()
        cells = 2048 * 1024
        out.append({"law": law, "value": cells * 50 / (t1 - t0), "unit": UNIT, "ms_per_step": (t1 - t0) / 50 * 1e3,
                    "newton_updates_per_solve": its / (70 * ((2049 * 1024) + (2048 * 1025)))})
    return {"workload": "antidune physics 2048x1024 (24 x 12 m), FP64, per transport law", "steps": 50,
            "time": "wall clock around one host-synchronous sve_step call", "laws": out}


def crop(w, nx, ny):
    """The first ny rows and nx columns of a 2D workload (the same cells,
    physics and boundary types, the domain lengths scaled with the grid)."""
    p = w["params"]
    p2 = dict(p, nx=nx, ny=ny, lx=p["lx"] * nx / p["nx"], ly=p["ly"] * ny / p["ny"])
    return dict(w, params=p2, **{k: np.ascontiguousarray(w[k][:ny, :nx]) for k in ("h", "hu", "hv", "z")})


def run_fp32_error(args, sve, W, torch):
    """Error of the FP32-state path per config, against the FP64 path from
    the same initial state (the FP64 path equals the FP64 oracle to 1e-10
    relative, tested): the 2D dune (1024 x 512) for its 2000 steps, the 2D
    antidune on its full 8192 x 4096 grid for 200 steps and on a 1024 x 512
    crop of it (the same cells) for its 1000 steps.  Per field: relative
    L-infinity (max |d| / max |ref|) and relative L1 (sum |d| / sum |ref|);
    discharges are scaled by the largest discharge."""
    out = []
    anti = W.antidune2d()
    for name, w, n in (("2D dune 1024x512, 2000 steps (full run)", W.dune2d(), 2000),
                       ("2D antidune 8192x4096 (full grid), 200 steps", anti, 200),
                       ("2D antidune, 1024x512 crop of the 8192x4096 grid, 1000 steps (full run)",
                        crop(anti, 1024, 512), 1000)):
        res = {}
        for prec in ("fp64", "fp32"):
            s = sve.Solver(w["params"], prec)
            s.set_state(w["h"], w["hu"], w["hv"], w["z"])
            t = s.step(n)
            res[prec] = dict(s.get_state(), t=t)
            s.close()
        a, b = res["fp32"], res["fp64"]
        qs = max(float(np.max(np.abs(b["hu"]))), float(np.max(np.abs(b["hv"]))))
        errs = {}
        for k in ("h", "hu", "hv", "z"):
            d = np.abs(a[k].astype(np.float64) - b[k])
            linf_scale = qs if k in ("hu", "hv") else float(np.max(np.abs(b[k])))
            l1_scale = float(np.sum(np.abs(b["hu"])) + np.sum(np.abs(b["hv"]))) if k in ("hu", "hv") else float(np.sum(np.abs(b[k])))
            errs[k] = {"linf": float(np.max(d)) / linf_scale, "l1": float(np.sum(d)) / l1_scale}
        out.append({"workload": name, "steps": n, "errors": errs, "t_fp64": b["t"], "t_fp32": a["t"]})
    return out


def advance_to(s, T, chunk=2000):
    """CFL steps until the simulated time reaches T exactly: bulk steps while
    more than two CFL steps remain, single steps after that, and a last
    fixed step with the remaining time once it is below the last CFL step
    (the CFL step changes little from one step to the next).  Returns the
    number of steps."""
    n = 0
    while True:
        d = s.diag()
        rest = T - d["t"]
        if rest <= 0.0:
            return n
        if n == 0:
            s.step(1)
            n = 1
            continue
        dt = d["dt"]
        if rest <= 0.99 * dt:
            s.step_dt(np.array([rest]))
            return n + 1
        k = int(rest / dt) - 2
        if k >= 1:
            k = min(k, chunk)
            s.step(k)
            n += k
        else:
            s.step(1)
            n += 1


def run_paper_bump(args, sve, W, torch):
    """The 2D bump of Sec. 5.3 at the paper's resolution (4000 x 4000 over
    1000 x 1000 m, q0 = 10, 2D Grass m_g = 3): A_g = 1 to T = 500 s (and
    with --paper-bump2d A_g = 0.1 to T = 1000 s) in FP32 state, wall clock of
    the whole run, and the FP64 step at full size over 200 steps from the
    developed flow at T = 500 s.  The paper's own timings are in a stripped
    figure: no comparison number exists."""
    out = []
    x = (np.arange(4000) + 0.5) * 0.25

    def centroid(z):
        dz = np.clip(np.asarray(z, np.float64) - 0.1, 0.0, None)
        return float(np.sum(dz * x[None, :]) / max(float(np.sum(dz)), 1e-300))

    developed = None
    for A_g, T in ((1.0, 500.0), (0.1, 1000.0)) if args.paper_bump2d else ((1.0, 500.0),):
        w = W.paper_bump2d(A_g=A_g)
        s = sve.Solver(w["params"], "fp32")
        s.set_state(w["h"], w["hu"], w["hv"], w["z"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = advance_to(s, T)
        wall = time.perf_counter() - t0
        st = s.get_state()
        t_end = s.diag()["t"]
        s.close()
        if developed is None:
            developed = st
        out.append({"A_g": A_g, "T": T, "precision": "fp32", "steps": n, "t_end": t_end, "wall_s": wall,
                    "value": 16e6 * n / wall, "unit": UNIT,
                    "bump_centroid_x_m": [centroid(w["z"]), centroid(st["z"])],
                    "z_max_m": [float(np.max(w["z"])), float(np.max(st["z"]))]})
    # FP64 from the developed flow at T = 500 s (A_g = 1): early steps are
    # not representative, most neighbours are still identical there and
    # their interfaces need no solve
    w = W.paper_bump2d(A_g=1.0)
    s = sve.Solver(w["params"], "fp64")
    s.set_state(*(developed[k].astype(np.float64) for k in ("h", "hu", "hv", "z")))
    s.step(20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.step(200)
    wall = time.perf_counter() - t0
    dt = s.diag()["dt"]
    s.close()
    out.append({"A_g": 1.0, "precision": "fp64", "steps": 200, "from": "the FP32 state at T = 500 s",
                "value": 16e6 * 200 / wall, "unit": UNIT, "ms_per_step": wall / 200 * 1e3, "cfl_dt_s": dt,
                "T500_estimate_s": 500.0 / dt * wall / 200})
    return {"workload": "2D bump (Sec. 5.3), 4000 x 4000 cells over 1000 x 1000 m", "runs": out,
            "time": "wall clock around host-synchronous sve_step calls"}


def measure_step(sve, torch, w, prec, local, world, spinup, warmup, steps, clocks=False):
    """Device time of `steps` single steps of workload w in precision prec,
    after `spinup` untimed steps and `warmup` warm-up steps: each step
    between CUDA events on the solver's stream, an L2 flush (a 256 MiB
    write) before each outside the events, the kernels' own event times from
    the library's profiling, the Newton counter over the timed steps; time
    max over ranks.  Returns the open solver with the numbers."""
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    stream = torch.cuda.current_stream()
    solver = sve.Solver(w["params"], prec, stream=stream.cuda_stream)
    solver.set_state(w["h"], w["hu"], w["hv"], w["z"])
    # spin-up: the first steps of a run can be cheaper (neighbours that are
    # still identical skip their solves); advance into the regime of the run
    if spinup > 0:
        solver.step(spinup)
    for _ in range(warmup):
        solver.step(1)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    c0 = solver.counters()
    solver.profile(True)
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        sampler.start()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_start()
    for k in range(steps):
        flush.zero_()                      # L2 flush between timed steps (outside the events)
        ev[k][0].record(stream)
        solver.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_end()
    if world > 1:
        dist.barrier()
    clk = sampler.stop() if sampler else None
    solver.sync()
    total_ms = float(np.sum([a.elapsed_time(b) for a, b in ev]))
    prof = solver.profile_read()
    solver.profile(False)
    c1 = solver.counters()
    if world > 1:
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    del flush
    return {"solver": solver, "value": world * nx * ny * steps / (total_ms * 1e-3), "ms_per_step": total_ms / steps,
            "prof": prof, "newton": c1["newton_iters"] - c0["newton_iters"], "steps": steps, "clocks": clk,
            "timed_steps_of_run": f"{spinup + warmup}..{spinup + warmup + steps - 1}"}


def measure_call(sve, torch, w, prec, spinup, warmup, steps):
    """Device time of one call of `steps` steps (sve_step_async(steps)
    between CUDA events on the solver's stream; for a grid whose state is
    larger than L2, so no flush is needed between its steps): the FP32 2D
    state's carried update runs within such a call.  The kernels' times
    from a second, profiled call of as many steps; the Newton counter over
    the timed call."""
    stream = torch.cuda.current_stream()
    solver = sve.Solver(w["params"], prec, stream=stream.cuda_stream)
    solver.set_state(w["h"], w["hu"], w["hv"], w["z"])
    if spinup > 0:
        solver.step(spinup)
    for _ in range(warmup):
        solver.step(1)
    c0 = solver.counters()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    solver.step_async(steps)
    b.record(stream)
    torch.cuda.synchronize()
    solver.sync()
    total_ms = a.elapsed_time(b)
    c1 = solver.counters()
    solver.profile(True)
    solver.step_async(steps)
    solver.sync()
    prof = solver.profile_read()
    solver.profile(False)
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    return {"solver": solver, "value": nx * ny * steps / (total_ms * 1e-3), "ms_per_step": total_ms / steps,
            "prof": prof, "newton": c1["newton_iters"] - c0["newton_iters"], "steps": steps, "clocks": None,
            "timed_steps_of_run": f"{spinup + warmup}..{spinup + warmup + steps - 1}"}


def march_shape(nx, ny, nsm=None):
    """Strips and runs of rows of the FP32 solve pass for a grid (the launch
    shape the library picks: 30 columns a strip, rows a run so that every SM
    has its 20 resident warps, 4 to 32)."""
    if nsm is None:
        import torch

        nsm = torch.cuda.get_device_properties(0).multi_processor_count
    strips = -(-nx // 30)
    rows = min(32, max(4, -(-(strips * ny) // (20 * nsm))))
    return strips, -(-ny // rows)


def roofline_of(m, w, prec, traffic_ok=False):
    """Roofline of the dominant kernel of a measured step (measure_step):
    FP64 -- interface_kernel<double>, bound by the FP64 ALUs: algorithmic
    FLOP per interface (setup, evaluations and updates by the device's Newton
    counter, final states and fluctuations) x interfaces / its mean event
    time, against the nominal FP64 rate; FP32 in 2D -- march_kernel<float>,
    the same count per interface (the Newton counter over the solves done,
    which include the strips' shared edges and one row per run of rows)
    against the nominal FP32 rate.
    Both give the step's algorithmic HBM fraction (64 / 32 B per cell)."""
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    cells = nx * ny
    steps = m["steps"]
    prof = m["prof"]
    n_iface = (nx + 1) * ny + nx * (ny + 1)
    iface_ms = prof["iface_ms"] / max(prof["iface_launches"], 1)
    cell_ms = prof["cell_ms"] / max(prof["cell_launches"], 1)
    hbm = peaks().get("hbm_gbs", 6800.3)
    bytes_per_cell = BYTES_PER_CELL_FP64 if prec == "fp64" else BYTES_PER_CELL_FP64 // 2
    step_frac = (bytes_per_cell * cells / (m["ms_per_step"] * 1e-3)) / (hbm * 1e9)
    if prec == "fp32":
        strips, chunks = march_shape(nx, ny)
        solves = ny * (nx + strips - 1) + nx * (ny + chunks)
        upd = m["newton"] / (solves * steps)
        flop = FLOP_SETUP + (1 + upd) * FLOP_EVAL + upd * FLOP_UPDATE + FLOP_FINAL
        ach = n_iface * flop / (iface_ms * 1e-3)
        return {"bound": "alu", "achieved": ach / 1e12, "peak": FP32_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_FLOPS, "traffic": None, "kernel": "march_kernel<float>",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (nominal FP32 FMA rate)",
                "flop_per_interface": flop, "newton_updates_per_solve": upd,
                "iface_ms": iface_ms, "cell_ms": cell_ms, "apply_launches": prof["cell_launches"],
                "hbm_frac_of_step": step_frac, "hbm_peak_gbs": hbm}
    upd = m["newton"] / (n_iface * steps)
    flop = FLOP_SETUP + (1 + upd) * FLOP_EVAL + upd * FLOP_UPDATE + FLOP_FINAL
    ach = n_iface * flop / (iface_ms * 1e-3)
    r = {"bound": "alu", "achieved": ach / 1e12, "peak": FP64_PEAK_FLOPS / 1e12, "unit": "TFLOP/s",
         "frac": ach / FP64_PEAK_FLOPS, "traffic": iface_traffic() if traffic_ok else None,
         "kernel": "interface_kernel<double>", "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
         "(GB300 FP64 nominal 1.25 TFLOP/s); a measured DFMA loop gave 1.19 TFLOP/s",
         "flop_per_interface": flop, "newton_updates_per_solve": upd,
         "iface_ms": iface_ms, "cell_ms": cell_ms, "hbm_frac_of_step": step_frac, "hbm_peak_gbs": hbm}
    if r["traffic"]:
        # the kernel's DRAM throughput from its ncu byte count and its event time
        r["dram_gbs"] = r["traffic"] / (iface_ms * 1e-3) / 1e9
        r["dram_frac"] = r["dram_gbs"] / hbm
    return r


def run_c3(args, sve, W, torch, local):
    """The largest config: the 2D antidune, 8192 x 4096 cells (24 x 12 m,
    supercritical inflow, random bed, MPM + Darcy), FP64 and FP32 state,
    after 30 untimed steps of the run, with the roofline of each form's
    dominant kernel: FP64 device-timed like the headline (L2 flush between
    single steps, CUDA events); FP32 as one call of its steps (its state,
    1 GB with the fluctuation planes, is far larger than L2), within which
    each step's solve pass applies the previous step's update."""
    w = W.antidune2d()
    out = {"workload": workload_desc(8192, 4096, "antidune2d", "fp64/fp32"), "nx": 8192, "ny": 4096}
    for prec, steps in (("fp64", args.c3_steps_fp64), ("fp32", args.c3_steps_fp32)):
        if prec == "fp64":
            m = measure_step(sve, torch, w, prec, local, 1, 30, 3, steps)
        else:
            m = measure_call(sve, torch, w, prec, 30, 3, steps)
        m["solver"].close()
        out[prec] = {"value": m["value"], "unit": UNIT, "ms_per_step": m["ms_per_step"], "steps": steps,
                     "timed_steps_of_run": m["timed_steps_of_run"], "roofline": roofline_of(m, w, prec),
                     "gpu_launches": int(m["prof"]["iface_launches"] + m["prof"]["cell_launches"])}
        if prec == "fp32":
            out[prec]["timing"] = ("one sve_step_async call of all steps between CUDA events (no L2 flush: "
                                   "1 GB state); the solve pass of each step but the first applies the "
                                   "previous step's update, one apply pass after the last")
    out["fp32_vs_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    return out


def run_plain_fp32(args, sve, W, torch, local):
    """The plain single-run step of the 2D dune in FP32 state (the batched
    FP32 ensemble's C2 physics is compared with it), device-timed as the
    headline over the same window of the run."""
    w = W.dune2d()
    m = measure_step(sve, torch, w, "fp32", local, 1, args.spinup, args.warmup, min(args.steps, 200))
    m["solver"].close()
    return {"workload": workload_desc(1024, 512, "dune2d", "fp32"), "value": m["value"], "unit": UNIT,
            "ms_per_step": m["ms_per_step"], "timed_steps_of_run": m["timed_steps_of_run"],
            "roofline": roofline_of(m, w, "fp32")}


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1307_0491_gb300 import build as B
    from paper_1307_0491_gb300 import sve
    from paper_1307_0491_gb300 import workloads as W

    B.build()
    w = make_workload(args, W, seed=rank)
    nx, ny = w["params"]["nx"], w["params"]["ny"]
    cells = nx * ny
    prec = args.precision
    stream = torch.cuda.current_stream()
    m = measure_step(sve, torch, w, prec, local, world, args.spinup, args.warmup, args.steps, clocks=True)
    solver, value, ms_per_step, prof, clk = m["solver"], m["value"], m["ms_per_step"], m["prof"], m["clocks"]
    roofline = roofline_of(m, w, prec, traffic_ok=(prec == "fp64" and args.workload == "dune2d" and not args.nx))

    # end to end through the C ABI from pinned host memory: every step uploads
    # the state reached by the timed steps (the same regime as `value`),
    # steps once and reads the new state back
    e2e_steps = min(args.steps, 50)
    npdt = np.float64 if prec == "fp64" else np.float32
    st = solver.get_state()
    host_in = {k: torch.from_numpy(np.ascontiguousarray(st[k], dtype=npdt)).pin_memory() for k in ("h", "hu", "hv", "z")}
    host_out = {k: torch.empty_like(host_in[k]).pin_memory() for k in host_in}
    ptr = {k: host_in[k].data_ptr() for k in host_in}
    optr = {k: host_out[k].data_ptr() for k in host_out}
    keys = ("h", "hu", "hv", "z")
    inp, outp = [ptr[k] for k in keys], [optr[k] for k in keys]

    def e2e_advance():
        rc, _ = sve.sve_advance(solver.h, 1, inp, outp, sve.SVE_HOST)
        if rc:
            raise sve.SveError(rc, "e2e step")

    def e2e_three_calls():
        rc = sve.sve_set_state(solver.h, *inp, sve.SVE_HOST)
        rc = rc or sve.sve_step(solver.h, 1)[0]
        rc = rc or sve.sve_get_state(solver.h, *outp, sve.SVE_HOST)
        if rc:
            raise sve.SveError(rc, "e2e step")

    def e2e_time(fn):
        fn()  # first call: page-locked buffer lookups, launch set-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            fn()
        secs = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([secs], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            secs = float(t.item())
        return secs

    e2e_s = e2e_time(e2e_advance)
    e2e_s3 = e2e_time(e2e_three_calls)
    io_bytes = 4 * (8 if prec == "fp64" else 4) * cells
    e2e = {"value": world * cells * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
           "d2h_bytes_per_step": io_bytes, "steps": e2e_steps,
           "call": "sve_advance(1 step) from and to page-locked host buffers, one call per step",
           "three_calls_value": world * cells * e2e_steps / e2e_s3}
    solver.close()

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32 (FP64 dt, t, mass sums)",
            "data": "synthetic",
            "config": bench_config(args, nx, ny),
            "roofline": roofline,
            "e2e": e2e,
            "gpu_launches": int(prof["iface_launches"] + prof["cell_launches"]),
            "clocks": clk,
        }
        plain32 = None
        if not args.no_c3:
            line["c3"] = run_c3(args, sve, W, torch, local)
        if not args.no_batch or not args.no_c3:
            plain32 = run_plain_fp32(args, sve, W, torch, local)
            line["plain_fp32_c2"] = plain32
        if not args.no_batch:
            line["batched"] = [run_batched(args, sve, W, torch, "fp64", value)]
            if not args.no_batch_fp32:
                line["batched"].append(run_batched(args, sve, W, torch, "fp32", plain32["value"]))
        if not args.no_adjoint:
            line["adjoint"] = run_adjoint(args, sve, W, torch)
        if not args.no_small1d:
            line["small1d"] = run_small1d(args, sve, W, torch)
            line["splitting"] = run_splitting(args, sve, W, torch)
        if not args.no_closures:
            line["closures"] = run_closures(args, sve, W, torch)
        if not args.no_fp32_error:
            line["fp32_error"] = run_fp32_error(args, sve, W, torch)
        if not args.no_paper_bump2d:
            line["paper_bump2d"] = run_paper_bump(args, sve, W, torch)
        if world == 1 and not args.no_cpu_baseline:
            from oracle.banded import host_threads

            cores = host_threads()
            # the oracle's own run to the window the GPU arm timed (its
            # spin-up and warm-up steps, untimed), then timed steps from there
            spun = oracle_spinup(w, cores, args.spinup + args.warmup)
            rate, nsteps, secs = cpu_oracle_rate(w, cores, state=spun)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"full {nx}x{ny} grid, {nsteps} step(s) in {secs:.1f} s from step "
                                              f"{args.spinup + args.warmup} of the run, C oracle on {cores} "
                                              f"threads (row bands of its block API)"}
            rate1, nsteps1, secs1 = cpu_oracle_rate(w, 1, state=spun)
            line["cpu_baseline"]["single_thread"] = {
                "value": rate1, "cores": 1,
                "sample": f"full {nx}x{ny} grid, {nsteps1} step(s) in {secs1:.1f} s from step "
                          f"{args.spinup + args.warmup} of the run, single-threaded C oracle"}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--spinup", type=int, default=400, help="untimed steps before warm-up (run regime)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble measurement")
    ap.add_argument("--batch-runs", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--batch-spinup", type=int, default=100)
    ap.add_argument("--no-batch-fp32", action="store_true", help="skip the FP32-state ensemble")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-small1d", action="store_true", help="skip the small-1D measurement")
    ap.add_argument("--no-closures", action="store_true", help="skip the per-transport-law measurement")
    ap.add_argument("--paper-bump2d", action="store_true",
                    help="the 2D bump of Sec. 5.3 at 4000 x 4000 also with A_g = 0.1 to T = 1000 s (FP32; +2 min)")
    ap.add_argument("--no-paper-bump2d", action="store_true",
                    help="skip the 2D bump of Sec. 5.3 at 4000 x 4000 (A_g = 1 to T = 500 s in FP32, then 200 "
                         "FP64 steps from there; ~1 min)")
    ap.add_argument("--no-fp32-error", action="store_true",
                    help="skip the FP32-state error per config")
    ap.add_argument("--no-c3", action="store_true", help="skip the 8192 x 4096 antidune (FP64 and FP32)")
    ap.add_argument("--c3-steps-fp64", type=int, default=20)
    ap.add_argument("--c3-steps-fp32", type=int, default=100)
    ap.add_argument("--workload", choices=["dune2d", "antidune2d"], default="dune2d")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--nx", type=int, default=0, help="grid override (profiling captures)")
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--adjoint-steps", type=int, default=4000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
