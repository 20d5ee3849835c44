"""The domain decomposition the path would use on several GPUs (Sec. 4: split
the grid into blocks, exchange one ghost layer per step), checked on the CPU
with two gloo ranks: each rank steps its block of the oracle grid, the ranks
exchange their boundary rows/columns and max-reduce the wave speeds for the
CFL step, and the gathered result equals the undecomposed oracle run bit for
bit.  (The GPU kernels are single-device here; this pins the sharded design:
its halo width, the ghost rules on physical sides and the global time step.)
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import oracle
from paper_1307_0491_gb300 import workloads as W

FIELDS = ("h", "hu", "hv", "z")
SIDES = {"W": 0, "E": 1, "S": 2, "N": 3}


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name: str):
    if name == "x_periodic":
        w = W.random_smooth(48, 20, seed=31, bc=("periodic", "periodic", "wall", "free"), A_g=0.05,
                            friction="strickler", K_st=30.0)
        return w, "x"
    if name == "y_inflow":
        w = W.dune2d(nx=40, ny=36, seed=32, lx=40.0, ly=36.0)
        w["params"].update(bc=("inflow_q", "free", "wall", "free"))
        return w, "y"
    w = W.antidune2d(nx=50, ny=24, seed=33)
    return w, "x"


def _worker(rank: int, world: int, port: int, case: str, nsteps: int, out_path: str):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, axis = _case(case)
    p = w["params"]
    P = oracle.Params.from_workload(p)
    orc = oracle.get()
    nx, ny = p["nx"], p["ny"]
    if axis == "x":
        cut = nx // 2
        x0, x1 = (0, cut) if rank == 0 else (cut, nx)
        y0, y1 = 0, ny
    else:
        cut = ny // 2
        y0, y1 = (0, cut) if rank == 0 else (cut, ny)
        x0, x1 = 0, nx
    blk = oracle.Block(orc, P, x1 - x0, y1 - y0)
    blk.set_interior(*[np.asarray(w[k])[y0:y1, x0:x1] for k in FIELDS])
    other = 1 - rank
    periodic = (p["bc"][0] == "periodic") if axis == "x" else (p["bc"][2] == "periodic")
    dts = []
    for _ in range(nsteps):
        F = blk.f
        # halo exchange of one layer with the neighbour (both sides if periodic)
        if axis == "x":
            mine_hi = np.stack([F[k][1:-1, -2] for k in FIELDS])   # my last column
            mine_lo = np.stack([F[k][1:-1, 1] for k in FIELDS])    # my first column
        else:
            mine_hi = np.stack([F[k][-2, 1:-1] for k in FIELDS])   # my last row
            mine_lo = np.stack([F[k][1, 1:-1] for k in FIELDS])
        send_hi = torch.from_numpy(np.ascontiguousarray(mine_hi))
        send_lo = torch.from_numpy(np.ascontiguousarray(mine_lo))
        recv_a = torch.empty_like(send_hi)
        recv_b = torch.empty_like(send_hi)
        # rank 0 sends its high edge to rank 1 (rank 1's low ghost) and, if
        # periodic, its low edge (rank 1's high ghost); rank 1 mirrors it
        reqs = []
        if rank == 0:
            reqs.append(dist.isend(send_hi, other, tag=1))
            reqs.append(dist.irecv(recv_a, other, tag=2))
            if periodic:
                reqs.append(dist.isend(send_lo, other, tag=3))
                reqs.append(dist.irecv(recv_b, other, tag=4))
        else:
            reqs.append(dist.irecv(recv_a, other, tag=1))
            reqs.append(dist.isend(send_lo, other, tag=2))
            if periodic:
                reqs.append(dist.irecv(recv_b, other, tag=3))
                reqs.append(dist.isend(send_hi, other, tag=4))
        for r in reqs:
            r.wait()
        ra, rb = recv_a.numpy(), recv_b.numpy()
        for c, k in enumerate(FIELDS):
            if axis == "x":
                if rank == 0:
                    F[k][1:-1, -1] = ra[c]
                    if periodic:
                        F[k][1:-1, 0] = rb[c]
                else:
                    F[k][1:-1, 0] = ra[c]
                    if periodic:
                        F[k][1:-1, -1] = rb[c]
            else:
                if rank == 0:
                    F[k][-1, 1:-1] = ra[c]
                    if periodic:
                        F[k][0, 1:-1] = rb[c]
                else:
                    F[k][0, 1:-1] = ra[c]
                    if periodic:
                        F[k][-1, 1:-1] = rb[c]
        # physical sides of this block: the boundary rules
        if axis == "x":
            phys = ["S", "N"] + ([] if periodic else (["W"] if rank == 0 else ["E"]))
        else:
            phys = ["W", "E"] + ([] if periodic else (["S"] if rank == 0 else ["N"]))
        for side in phys:
            if p["bc"][SIDES[side]] != "periodic":
                blk.ghost(SIDES[side])
        if axis == "x" and p["bc"][2] == "periodic" or axis == "y" and p["bc"][0] == "periodic":
            raise RuntimeError("case not supported by this test")
        # global CFL step: max of the wave speeds over both blocks
        Sx, Sy = blk.speeds()
        S = torch.tensor([Sx, Sy], dtype=torch.float64)
        dist.all_reduce(S, op=dist.ReduceOp.MAX)
        dt = blk.dt(float(S[0]), float(S[1]))
        dts.append(dt)
        blk.advance(dt)
    np.savez(out_path + f".{rank}.npz", **{k: blk.interior(k) for k in FIELDS}, dts=np.array(dts),
             box=np.array([x0, x1, y0, y1]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", ["x_periodic", "y_inflow", "x_antidune"])
def test_two_rank_decomposition_equals_single_grid(case, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    nsteps = 25
    out = str(tmp_path / "blk")
    mp.start_processes(_worker, args=(2, _free_port(), case, nsteps, out), nprocs=2, join=True,
                       start_method="spawn")
    w, _ = _case(case)
    ref = oracle.get().run(oracle.Params.from_workload(w["params"]), nsteps, w["h"], w["hu"], w["hv"], w["z"])
    got = {k: np.zeros_like(np.asarray(w[k])) for k in FIELDS}
    dts = []
    for r in range(2):
        d = np.load(out + f".{r}.npz")
        x0, x1, y0, y1 = d["box"]
        for k in FIELDS:
            got[k][y0:y1, x0:x1] = d[k]
        dts.append(d["dts"])
    assert np.array_equal(dts[0], dts[1]) and np.array_equal(dts[0], ref["dts"])
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
