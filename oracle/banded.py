"""The FP64 oracle on all host cores: the 2D grid cut into bands of rows, one
padded block of the oracle's domain-decomposition API (Sec. 4: blocks with
one ghost layer) per band, stepped on a pool of threads.

Test infrastructure, like the rest of ``oracle/``: only the tests and the
benchmark's CPU legs use it.  It adds no arithmetic of its own: each band
runs the oracle's own block functions (``orc_block_ghost``,
``orc_block_solve``, ``orc_block_dt``, ``orc_block_update``), which do the
arithmetic of the whole-grid stepper, and the ctypes calls release the GIL,
so the bands run in parallel.  Per step: (1) every band's halo rows are
copied from its neighbours' interiors (periodic sides wrap), (2) each band
fills its ghosts on physical sides, solves its interfaces and returns its
extreme wave speeds, (3) the global CFL step is taken from the maximum over
the bands (an order-free reduction), (4) each band advances with the
fluctuations of its solve.  The result equals the
single-threaded run bit for bit (tested).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import BC_PERIODIC

FIELDS = ("h", "hu", "hv", "z")


def host_threads() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - platforms without affinity
        return os.cpu_count() or 1


class BandedRun:
    """A 2D oracle grid split into ``nbands`` bands of rows (sizes differ by
    at most one row), stepped on ``threads`` threads."""

    def __init__(self, orc, p, h, hu, hv, z, nbands: int | None = None, threads: int | None = None):
        from . import Block

        if p.dim != 2:
            raise ValueError("banded oracle: 2D grids only")
        self.p = p
        nb = int(nbands or host_threads())
        nb = max(1, min(nb, p.ny))
        self.threads = int(threads or nb)
        edges = [round(b * p.ny / nb) for b in range(nb + 1)]
        self.rows = [(edges[b], edges[b + 1]) for b in range(nb)]
        self.blocks = []
        fields = [np.asarray(a, dtype=np.float64).reshape(p.ny, p.nx) for a in (h, hu, hv, z)]
        for y0, y1 in self.rows:
            blk = Block(orc, p, p.nx, y1 - y0)
            blk.set_interior(*[f[y0:y1] for f in fields])
            self.blocks.append(blk)
        self.periodic_x = int(p.bc[0]) == BC_PERIODIC
        self.periodic_y = int(p.bc[2]) == BC_PERIODIC
        self.phys = []
        for b in range(nb):
            sides = [] if self.periodic_x else [0, 1]
            if not self.periodic_y:
                if b == 0:
                    sides.append(2)
                if b == nb - 1:
                    sides.append(3)
            self.phys.append(sides)
        self.pool = ThreadPoolExecutor(max_workers=self.threads)
        self.t = 0.0
        self.dts: list[float] = []

    def close(self):
        self.pool.shutdown(wait=True)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _halos(self):
        nb = len(self.blocks)
        for b, blk in enumerate(self.blocks):
            below = b - 1 if b > 0 else (nb - 1 if self.periodic_y else None)
            above = b + 1 if b < nb - 1 else (0 if self.periodic_y else None)
            for k in FIELDS:
                F = blk.f[k]
                if below is not None:
                    F[0, 1:-1] = self.blocks[below].f[k][-2, 1:-1]
                if above is not None:
                    F[-1, 1:-1] = self.blocks[above].f[k][1, 1:-1]
                if self.periodic_x:
                    F[1:-1, 0] = F[1:-1, -2]
                    F[1:-1, -1] = F[1:-1, 1]

    def _ghosts_and_speeds(self, b):
        blk = self.blocks[b]
        for side in self.phys[b]:
            blk.ghost(side)
        return blk.speeds()

    def step(self, nsteps: int = 1):
        for _ in range(nsteps):
            self._halos()
            S = list(self.pool.map(self._ghosts_and_speeds, range(len(self.blocks))))
            Sx = max(s[0] for s in S)
            Sy = max(s[1] for s in S)
            dt = self.blocks[0].dt(Sx, Sy)
            list(self.pool.map(lambda blk: blk.advance(dt), self.blocks))
            self.t += dt
            self.dts.append(dt)

    def state(self) -> dict:
        return {k: np.concatenate([blk.interior(k) for blk in self.blocks], axis=0) for k in FIELDS}
