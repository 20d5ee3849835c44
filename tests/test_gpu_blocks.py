"""The domain decomposition of Sec. 4 through the library's block calls
(sve_block_get_edge / sve_block_set_ghosts / sve_block_speeds /
sve_block_advance): a grid cut into blocks, each block a handle whose sides
toward the other blocks are SVE_BC_EXTERNAL, one ghost layer exchanged per
step through host buffers, the time step from the maximum of the blocks'
wave speeds.  The decomposed GPU run equals the whole-grid GPU run bit for
bit (same launch shape of the two-kernel step; the FP32 2D fused step too):
with the blocks in one process, and with two gloo ranks (two processes on
the one GPU, exchanging edges and max-reducing the speeds on the host; no
kernel waits on another process)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

from paper_1307_0491_gb300 import sve
from paper_1307_0491_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("h", "hu", "hv", "z")
W_, E_, S_, N_ = sve.SVE_W, sve.SVE_E, sve.SVE_S, sve.SVE_N


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()


def _case(name: str):
    if name == "x_periodic":
        w = W.random_smooth(96, 40, seed=31, bc=("periodic", "periodic", "wall", "free"), A_g=0.05,
                            friction="strickler", K_st=30.0)
        return w, "x"
    if name == "y_inflow":
        w = W.dune2d(nx=80, ny=72, seed=32, lx=80.0, ly=72.0)
        w["params"].update(bc=("inflow_q", "free", "wall", "free"), friction="strickler", K_st=40.0, q_in=0.5)
        return w, "y"
    if name == "x_collide":
        return W.colliding_streams(64, dim=2, ny=24, ymod=0.2), "x"
    return W.antidune2d(nx=100, ny=48, seed=33), "x"


def _blocks(w, axis: str, nb: int):
    """The blocks of a cut along axis into nb equal parts: their boxes
    (x0, x1, y0, y1), parameters (external sides toward the other blocks)
    and neighbours {side: (block, its side)}."""
    p = w["params"]
    nx, ny = p["nx"], p["ny"]
    dx, dy = p["lx"] / nx, p["ly"] / ny
    lo, hi = (W_, E_) if axis == "x" else (S_, N_)
    periodic = p["bc"][lo] == "periodic"
    n = nx if axis == "x" else ny
    cuts = [n * k // nb for k in range(nb + 1)]
    out = []
    for b in range(nb):
        a0, a1 = cuts[b], cuts[b + 1]
        box = (a0, a1, 0, ny) if axis == "x" else (0, nx, a0, a1)
        bc = list(p["bc"])
        nbrs = {}
        if b > 0 or periodic:
            bc[lo] = "external"
            nbrs[lo] = ((b - 1) % nb, hi)
        if b < nb - 1 or periodic:
            bc[hi] = "external"
            nbrs[hi] = ((b + 1) % nb, lo)
        q = dict(p, bc=tuple(bc), nx=box[1] - box[0], ny=box[3] - box[2], lx=(box[1] - box[0]) * dx,
                 ly=(box[3] - box[2]) * dy)
        out.append((box, q, nbrs))
    return out


def _cut(w, box):
    x0, x1, y0, y1 = box
    return {k: np.ascontiguousarray(np.asarray(w[k])[y0:y1, x0:x1]) for k in FIELDS}


def _whole(w, nsteps, precision):
    s = sve.Solver(w["params"], precision)
    if precision == "fp64":
        s.set_block_size(128)
    s.set_state(w["h"], w["hu"], w["hv"], w["z"])
    s.step(nsteps)
    out = s.get_state()
    out["dts"] = s.dts(nsteps)
    s.close()
    return out


@pytest.mark.parametrize("case,nb,precision", [
    ("x_periodic", 3, "fp64"), ("y_inflow", 2, "fp64"), ("x_antidune", 2, "fp64"), ("x_collide", 2, "fp64"),
    ("x_periodic", 2, "fp32"), ("y_inflow", 3, "fp32"),
])
def test_blocks_in_one_process_equal_whole_grid(case, nb, precision):
    w, axis = _case(case)
    nsteps = 40
    blocks = _blocks(w, axis, nb)
    hs = []
    for box, q, _ in blocks:
        s = sve.Solver(q, precision)
        if precision == "fp64":
            s.set_block_size(128)
        c = _cut(w, box)
        s.set_state(c["h"], c["hu"], c["hv"], c["z"])
        hs.append(s)
    dts = []
    for _ in range(nsteps):
        # each external side's ghosts from the neighbour's edge (interior
        # cells: untouched by setting ghosts, so the order does not matter)
        for b, (_, _, nbrs) in enumerate(blocks):
            for side, (ob, oside) in nbrs.items():
                hs[b].set_ghosts(side, hs[ob].edge(oside))
        sp = [s.block_speeds() for s in hs]
        sx, sy = max(v[0] for v in sp), max(v[1] for v in sp)
        for s in hs:
            s.block_advance(sx, sy)
        dts.append(float(hs[0].diag()["dt"]))
    got = {k: np.zeros_like(np.asarray(w[k]), dtype=np.float64 if precision == "fp64" else np.float32)
           for k in FIELDS}
    for (box, _, _), s in zip(blocks, hs):
        st = s.get_state()
        x0, x1, y0, y1 = box
        for k in FIELDS:
            got[k][y0:y1, x0:x1] = st[k]
        s.close()
    ref = _whole(w, nsteps, precision)
    assert np.array_equal(np.array(dts), ref["dts"])
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), (k, float(np.max(np.abs(got[k].astype(np.float64) - ref[k]))))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, case: str, nsteps: int, precision: str, out_path: str):
    """One gloo rank: its block as a handle on the GPU, its edges to the
    other rank through host tensors, the speeds max-reduced on the host."""
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1307_0491_gb300 import build

    build.build()
    sve.load()
    w, axis = _case(case)
    box, q, nbrs = _blocks(w, axis, world)[rank]
    s = sve.Solver(q, precision)
    if precision == "fp64":
        s.set_block_size(128)
    c = _cut(w, box)
    s.set_state(c["h"], c["hu"], c["hv"], c["z"])
    dts = []
    for _ in range(nsteps):
        # every external side sends its edge to the neighbour's opposite
        # side; receives are posted for the ghosts (world 2: one neighbour)
        reqs, recv = [], {}
        for side, (ob, oside) in sorted(nbrs.items()):
            send = torch.from_numpy(s.edge(side))
            recv[side] = torch.empty_like(send)
            reqs.append(dist.isend(send, dst=ob, tag=side))
            reqs.append(dist.irecv(recv[side], src=ob, tag=oside))
        for r in reqs:
            r.wait()
        for side, buf in recv.items():
            s.set_ghosts(side, buf.numpy())
        sx, sy = s.block_speeds()
        m = torch.tensor([sx, sy], dtype=torch.float64)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        s.block_advance(float(m[0]), float(m[1]))
        dts.append(float(s.diag()["dt"]))
    st = s.get_state()
    s.close()
    np.savez(out_path + f".{rank}.npz", **{k: st[k] for k in FIELDS}, dts=np.array(dts), box=np.array(box))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("case,precision", [("x_periodic", "fp64"), ("y_inflow", "fp64"), ("x_antidune", "fp32")])
def test_two_gloo_ranks_equal_whole_grid(case, precision, tmp_path):
    import torch.multiprocessing as mp

    nsteps = 30
    out = str(tmp_path / "blk")
    mp.start_processes(_rank, args=(2, _free_port(), case, nsteps, precision, out), nprocs=2, join=True,
                       start_method="spawn")
    w, _ = _case(case)
    ref = _whole(w, nsteps, precision)
    dtype = np.float64 if precision == "fp64" else np.float32
    got = {k: np.zeros(np.asarray(w[k]).shape, dtype=dtype) for k in FIELDS}
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
