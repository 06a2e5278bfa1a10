"""One grid split into slabs of rows across ranks, with a ghost-row exchange
per step and a max-reduction of the CFL wave speed.

This is the paper's Coarse-Grain decomposition (§3: one subdomain per
thread, neighbours exchanging boundary data) and its interface buffers (§5,
Fig. 10), with processes (one per GPU) in place of threads.  The grid's
rows are split into contiguous slabs, each of at least 2 rows.  A rank's
local grid is its slab plus 2 halo rows on each side that has a neighbour
(every side of a periodic y axis when there are several ranks); a side at
the grid's edge keeps the grid's own boundary condition, a halo side is
given a transmissive one, which only ever touches the halo rows.

A step, on every rank:
  1. exchange: the first two and the last two owned rows go to the
     neighbours, whose halo rows they become (two messages per neighbour
     per step, 2 rows x 4 variables x nx values each);
  2. dt: the local CFL step over all local cells -- owned and halo rows hold
     valid states now, and each halo row is some rank's owned row -- and the
     minimum over ranks, which is C h / (the global maximum wave speed)
     bit for bit (the correctly rounded quotient is monotone in the speed);
  3. one step of the scheme on the local grid with that dt, the sweep order
     set by the global step count.
The x sweep of a row reads only that row, so the halo rows swept along x
locally equal the neighbour's; the y sweep of an owned row reads at most two
rows on each side, all present.  The owned rows of every rank therefore
equal the same rows of the unsplit run bit for bit (the halo rows are
overwritten at the next exchange).  The backends are the library
(LibBackend, one hydro context per rank) or, in the tests, the CPU oracle;
communication is torch.distributed (gloo on CPU tensors, NCCL on CUDA
tensors) or, for several ranks in one process, direct hand-over
(step_in_process).  Nothing here computes any part of the scheme.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

REFLECT, TRANSMISSIVE, PERIODIC = 0, 1, 2
HALO = 2          # ghost rows per side (the stencil of Figs. 1-2)
TAG_UP, TAG_DOWN = 0, 1   # rows travelling to the next / previous rank


def split_rows(ny: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [j0, j1) of `world` slabs as equal as possible
    (the first ny % world get one more row); each holds at least 2 rows."""
    if world < 1 or ny < HALO * world:
        raise ValueError(f"cannot split {ny} rows into {world} slabs of at least {HALO} rows")
    base, extra = divmod(ny, world)
    out, j = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((j, j + n))
        j += n
    return out


@dataclass(frozen=True)
class Slab:
    """Rank `rank`'s part of a grid of ny rows: owned rows [j0, j1) and
    whether it has halo rows below j0 (lo) and above j1 (hi)."""
    rank: int
    world: int
    ny: int
    j0: int
    j1: int
    lo: bool
    hi: bool

    @property
    def owned(self) -> int:
        return self.j1 - self.j0

    @property
    def own0(self) -> int:
        """Local row index of global row j0."""
        return HALO if self.lo else 0

    @property
    def local_ny(self) -> int:
        return self.owned + HALO * (int(self.lo) + int(self.hi))

    def local_bc(self, bc) -> tuple:
        """Boundary conditions of the local grid: the grid's x conditions; y
        the grid's own at an edge, transmissive beside a halo."""
        return (bc[0], bc[1], TRANSMISSIVE if self.lo else bc[2], TRANSMISSIVE if self.hi else bc[3])

    def local_rows(self) -> np.ndarray:
        """Global row index of every local row."""
        rows = np.arange(self.j0 - (HALO if self.lo else 0), self.j1 + (HALO if self.hi else 0))
        return rows % self.ny


def slabs(ny: int, bc, world: int) -> list[Slab]:
    periodic = bc[2] == PERIODIC
    out = []
    for r, (j0, j1) in enumerate(split_rows(ny, world)):
        lo = world > 1 and (r > 0 or periodic)
        hi = world > 1 and (r < world - 1 or periodic)
        out.append(Slab(r, world, ny, j0, j1, lo, hi))
    return out


class SlabRank:
    """The host logic of one rank: which rows go where, and the step."""

    def __init__(self, slab: Slab, backend):
        self.slab = slab
        self.b = backend

    def outgoing(self) -> list[tuple[int, int, np.ndarray]]:
        """(destination rank, tag, rows [4, 2, nx]) of this step's messages."""
        s, msgs = self.slab, []
        if s.hi:  # my last two owned rows become the next rank's low halo
            msgs.append(((s.rank + 1) % s.world, TAG_UP, self.b.get_rows(s.own0 + s.owned - HALO, HALO)))
        if s.lo:  # my first two owned rows become the previous rank's high halo
            msgs.append(((s.rank - 1) % s.world, TAG_DOWN, self.b.get_rows(s.own0, HALO)))
        return msgs

    def incoming(self) -> list[tuple[int, int, int]]:
        """(source rank, tag, local row) of the halo rows this rank receives."""
        s, ins = self.slab, []
        if s.lo:
            ins.append(((s.rank - 1) % s.world, TAG_UP, 0))
        if s.hi:
            ins.append(((s.rank + 1) % s.world, TAG_DOWN, s.own0 + s.owned))
        return ins

    def receive(self, row0: int, rows) -> None:
        self.b.set_rows(row0, rows)

    def local_dt(self) -> float:
        return float(self.b.cfl_dt())

    def advance(self, dt: float) -> None:
        self.b.step(dt)

    def owned_state(self):
        s = self.slab
        return self.b.get_rows(s.own0, s.owned)


def step_in_process(ranks: list[SlabRank], nsteps: int) -> None:
    """Advance several ranks held by one process (each its own context),
    handing the messages over directly: the same steps as step_distributed,
    with no kernel ever waiting for another rank's."""
    for _ in range(nsteps):
        mail = {}
        for rk in ranks:
            for dst, tag, rows in rk.outgoing():
                mail[(rk.slab.rank, dst, tag)] = rows
        for rk in ranks:
            for src, tag, row0 in rk.incoming():
                rk.receive(row0, mail[(src, rk.slab.rank, tag)])
        dt = min(rk.local_dt() for rk in ranks)
        for rk in ranks:
            rk.advance(dt)


def step_distributed(rank: SlabRank, nsteps: int, dist, make_tensor=None) -> None:
    """Advance this process's rank with torch.distributed: point-to-point
    sends of the boundary rows, then one MIN all-reduce of dt per step.
    make_tensor(array) -> tensor places a message where the process group
    wants it (gloo: CPU tensors, the default; NCCL: CUDA tensors)."""
    import torch

    make_tensor = make_tensor or (lambda a: torch.as_tensor(np.ascontiguousarray(a)))
    for _ in range(nsteps):
        reqs, bufs, keep = [], [], []
        for src, tag, row0 in rank.incoming():
            t = make_tensor(np.zeros((4, HALO, rank.b.nx)))
            reqs.append(dist.irecv(t, src=src, tag=tag))
            bufs.append((row0, t))
        for dst, tag, rows in rank.outgoing():
            t = make_tensor(rows)
            keep.append(t)
            reqs.append(dist.isend(t, dst=dst, tag=tag))
        for r in reqs:
            r.wait()
        for row0, t in bufs:
            rank.receive(row0, t)
        dt = make_tensor(np.array([rank.local_dt()]))
        dist.all_reduce(dt, op=dist.ReduceOp.MIN)
        rank.advance(float(dt.cpu().numpy()[0]))


class LibBackend:
    """A rank's local grid in one hydro context (the library's kernels do
    every step of the scheme)."""

    def __init__(self, slab: Slab, nx: int, h: float, bc, U_local, precision: int = 64,
                 step0: int = 0, **ctx_kw):
        from . import hydro as H
        self.nx = nx
        self.ctx = H.Context([(nx, slab.local_ny, h, slab.local_bc(bc))], precision=precision, **ctx_kw)
        self.ctx.set_state(0, U_local)
        self.ctx.set_step(step0)

    def get_rows(self, row0: int, nrows: int):
        return self.ctx.get_rows(0, row0, nrows)

    def set_rows(self, row0: int, rows) -> None:
        # a CUDA tensor goes in as a device pointer, a CPU tensor as an array
        if hasattr(rows, "is_cuda") and not rows.is_cuda:
            rows = rows.numpy()
        self.ctx.set_rows(0, row0, rows)

    def cfl_dt(self) -> float:
        return self.ctx.cfl_dt(0)

    def step(self, dt: float) -> None:
        self.ctx.step(1, dt_override=np.array([dt]))

    def close(self) -> None:
        self.ctx.close()
