"""Row-slab domain decomposition of one grid over several ranks.

The two-step (Eq. A2) updates a node from the nodes within the stencil
radius R of it (the stencil Q_m of Section 4), and the first step (Eq. A1)
likewise.  A band of rows advanced T levels on its own is therefore exact
except in the R T rows nearest each of its edges.  A grid of ny rows split
into row slabs, each slab extended by H = R T halo rows on every side it
shares with another slab and refreshed from its neighbours after every T
levels, reproduces the undivided run bit for bit: every owned node goes
through the same per-node arithmetic on the same operand values.

One rank holds one slab (its local solver, e.g. a ``Wave2D`` handle of
nx x (owned + halo) rows on its GPU).  After the first step and after every
T levels the ranks exchange halo rows, both state planes (u^{k-1}, u^k):

* "up" messages carry a slab's top H owned rows to the rank above, into the
  bottom halo there; "down" messages its bottom H owned rows to the rank
  below, into the top halo there;
* every rank posts, in this order: send up, send down, receive from below
  (an up message), receive from above (a down message).  The order is the
  same on every rank, so messages between one pair of ranks match in the
  order they were posted (two ranks on a periodic grid are each other's
  upper and lower neighbour).

Zero boundary: the first and the last slab have no halo on their outer side
(the local solver's zero ring is the grid's boundary there).  Periodic: the
slabs form a ring.  A slab's local solver keeps the grid's boundary
condition; in the direction across slabs its own boundary (zero ring or
wrap) only touches halo rows, which the next exchange overwrites.

Norms (Eq. error): each rank reduces its owned rows (sums of squares and
maxima, wave2d_error_sums) and the ranks combine them with one sum and one
maximum over all ranks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

UP, DOWN = 0, 1  # message tags


@dataclass(frozen=True)
class SlabPlan:
    nx: int
    ny: int
    world: int
    rank: int
    R: int            # stencil radius
    T: int            # levels between exchanges
    periodic: bool
    r0: int           # owned global rows [r0, r1)
    r1: int
    lo_halo: int      # halo rows below the owned rows
    hi_halo: int      # halo rows above the owned rows
    down: Optional[int]
    up: Optional[int]

    @property
    def H(self) -> int:
        return self.R * self.T

    @property
    def own(self) -> int:
        return self.r1 - self.r0

    @property
    def ny_local(self) -> int:
        return self.lo_halo + self.own + self.hi_halo

    @property
    def e0(self) -> int:
        """Global row of local row 0 (negative for the first periodic slab)."""
        return self.r0 - self.lo_halo

    @property
    def owned_local(self) -> tuple[int, int]:
        return self.lo_halo, self.lo_halo + self.own

    def global_rows(self) -> np.ndarray:
        """Global row index of every local row (wrapped on periodic grids)."""
        g = np.arange(self.e0, self.e0 + self.ny_local)
        return g % self.ny if self.periodic else g

    def sends(self):
        """(peer, tag, first local row) of the messages this slab sends, in
        posting order; each carries H rows of both planes."""
        out = []
        lo, hi = self.owned_local
        if self.up is not None:
            out.append((self.up, UP, hi - self.H))
        if self.down is not None:
            out.append((self.down, DOWN, lo))
        return out

    def recvs(self):
        """(peer, tag, first local row) of the messages this slab receives,
        in posting order."""
        out = []
        if self.down is not None:
            out.append((self.down, UP, 0))
        if self.up is not None:
            out.append((self.up, DOWN, self.ny_local - self.H))
        return out


def plan_slabs(nx: int, ny: int, world: int, rank: int, R: int, T: int, periodic: bool) -> SlabPlan:
    """The slab of ``rank`` among ``world`` ranks: rows split as evenly as
    possible (the first ny mod world slabs one row taller), halos of R T rows.
    Every slab must own at least R T rows (its neighbours' halos come from it
    alone)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if R < 1 or T < 1:
        raise ValueError("stencil radius and levels per exchange must be >= 1")
    base, extra = divmod(ny, world)
    r0 = rank * base + min(rank, extra)
    r1 = r0 + base + (1 if rank < extra else 0)
    H = R * T
    if world == 1:
        return SlabPlan(nx, ny, 1, 0, R, T, periodic, 0, ny, 0, 0, None, None)
    if base < H:
        raise ValueError(f"{ny} rows over {world} ranks leave slabs of {base} rows, fewer than the "
                         f"{H} halo rows (R {R} x T {T}) a neighbour needs")
    if periodic:
        down, up = (rank - 1) % world, (rank + 1) % world
        lo, hi = H, H
    else:
        down = rank - 1 if rank > 0 else None
        up = rank + 1 if rank < world - 1 else None
        lo = H if down is not None else 0
        hi = H if up is not None else 0
    return SlabPlan(nx, ny, world, rank, R, T, periodic, r0, r1, lo, hi, down, up)


def extended_rows(plan: SlabPlan, field: np.ndarray) -> np.ndarray:
    """The slab's local rows (owned and halo) of a whole-grid field (ny x nx)."""
    return np.ascontiguousarray(field[plan.global_rows()])


def shard(items, rank: int, world: int):
    """Independent work (batched instances, served requests) split over the
    ranks round robin: rank r takes items r, r + world, ...  No exchange."""
    return list(items)[rank::world]


class SlabRun:
    """One slab: its plan, its local solver and the packing of its messages.

    ``solver`` is the local solver of the slab's ny_local rows; it provides
    first_step(u0, v0), step_n(n), get_rows(j0, n, prev, cur),
    set_rows(j0, n, prev, cur), row_block_shape(n) -> (shape, numpy dtype),
    error_sums(ex, j0, nrows, row_shift) and sync().  Message buffers are
    torch tensors on ``device`` (a CUDA device for NCCL, "cpu" for gloo)."""

    def __init__(self, plan: SlabPlan, solver, device="cpu"):
        self.plan = plan
        self.solver = solver
        self.device = device
        self.k = 0
        shape, dtype = solver.row_block_shape(max(plan.H, 1))
        self._msg_shape = (2,) + tuple(shape)
        self._np_dtype = dtype

    def _buffer(self):
        import torch
        td = torch.float64 if self._np_dtype == np.float64 else torch.float32
        return torch.empty(self._msg_shape, dtype=td, device=self.device)

    def outgoing(self, sync=True):
        """Pack the rows this slab sends: [(peer, tag, tensor of both planes)].
        ``sync``: wait for the copies (another stream, a communication
        library or the host reads the buffers next)."""
        out = []
        for peer, tag, j0 in self.plan.sends():
            buf = self._buffer()
            self.solver.get_rows(j0, self.plan.H, buf[0], buf[1])
            out.append((peer, tag, buf))
        if sync:
            self.solver.sync()  # device copies done before another stream reads them
        return out

    def incoming(self):
        """Buffers for the rows this slab receives: [(peer, tag, tensor)]."""
        return [(peer, tag, self._buffer()) for peer, tag, _ in self.plan.recvs()]

    def apply(self, received):
        """Unpack received rows into the halo (received in recvs() order)."""
        for (_, _, j0), (_, _, buf) in zip(self.plan.recvs(), received):
            self.solver.set_rows(j0, self.plan.H, buf[0], buf[1])

    def error_sums(self, ex):
        lo, hi = self.plan.owned_local
        return self.solver.error_sums(ex, lo, hi - lo, self.plan.e0)


def first_step(runs, exchange, u0s, v0s):
    """Eq. A1 on every slab's local rows (owned and halo), then a halo
    exchange: the first step leaves the R rows nearest each cut stale."""
    for r, u0, v0 in zip(runs, u0s, v0s):
        r.solver.first_step(u0, v0)
        r.k = 1
    exchange.run(runs)


def step_n(runs, exchange, n: int):
    """n two-steps (Eq. A2) of every slab: runs of at most T levels, a halo
    exchange after each."""
    if n < 0:
        raise ValueError("n must be >= 0")
    T = runs[0].plan.T
    while n > 0:
        m = min(T, n)
        for r in runs:
            r.solver.step_n(m)
            r.k += m
        exchange.run(runs)
        n -= m


def error_vs_exact(runs, exchange, ex):
    """(relative L2, relative L-infinity) of u^k over the whole grid."""
    s = exchange.combine_sums([r.error_sums(ex) for r in runs])
    return math.sqrt(s[0] / s[1]), s[2] / s[3]


def combine(sums_list):
    """Sums (0, 1) add, maxima (2, 3) take the largest."""
    s = [0.0, 0.0, 0.0, 0.0]
    for t in sums_list:
        s[0] += t[0]
        s[1] += t[1]
        s[2] = max(s[2], t[2])
        s[3] = max(s[3], t[3])
    return s


class DistExchange:
    """Halo exchange between processes over torch.distributed, one slab per
    rank (NCCL with device buffers, gloo with host buffers)."""

    def __init__(self, group=None):
        self.group = group

    def run(self, runs):
        import torch.distributed as dist
        (run,) = runs
        sends = run.outgoing()
        recvs = run.incoming()
        ops = [dist.P2POp(dist.isend, buf, peer, self.group, tag) for peer, tag, buf in sends]
        ops += [dist.P2POp(dist.irecv, buf, peer, self.group, tag) for peer, tag, buf in recvs]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if recvs and recvs[0][2].is_cuda:
            import torch
            torch.cuda.current_stream(recvs[0][2].device).synchronize()  # received before the handle's stream reads
        run.apply(recvs)

    def combine_sums(self, sums_list):
        import torch
        import torch.distributed as dist
        s = combine(sums_list)
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        a = torch.tensor([s[0], s[1]], dtype=torch.float64, device=dev)
        m = torch.tensor([s[2], s[3]], dtype=torch.float64, device=dev)
        dist.all_reduce(a, op=dist.ReduceOp.SUM, group=self.group)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=self.group)
        return [float(a[0]), float(a[1]), float(m[0]), float(m[1])]


class LocalExchange:
    """The same exchange among all slabs of a grid held by one process (for
    example every slab on one GPU): messages are matched by (sender,
    receiver, tag) in posting order and copied directly.

    ``sync=False`` when every slab's solver launches on the stream that
    allocates the message buffers (every handle and torch on the default
    stream of one device): the row copies are then ordered by that stream and
    the exchange waits for nothing on the host."""

    def __init__(self, sync=True):
        self.sync = sync

    def run(self, runs):
        mail = {}
        for r in runs:
            for peer, tag, buf in r.outgoing(sync=self.sync):
                mail.setdefault((r.plan.rank, peer, tag), []).append(buf)
        for r in runs:
            got = [(peer, tag, mail[(peer, r.plan.rank, tag)].pop(0)) for peer, tag, _ in r.plan.recvs()]
            r.apply(got)

    def combine_sums(self, sums_list):
        return combine(sums_list)


class HandleSolver:
    """Local solver of a slab: a ``Wave2D`` handle of nx x ny_local rows."""

    def __init__(self, sim):
        self.sim = sim

    def first_step(self, u0, v0):
        self.sim.first_step(u0, v0)

    def step_n(self, n):
        self.sim.step_n(n)

    def get_rows(self, j0, n, prev, cur):
        self.sim.get_rows(j0, n, prev, cur)

    def set_rows(self, j0, n, prev, cur):
        self.sim.set_rows(j0, n, prev, cur)

    def row_block_shape(self, n):
        return self.sim.row_block_shape(n)

    def error_sums(self, ex, j0, nrows, row_shift):
        return self.sim.error_sums(ex, j0, nrows, row_shift)

    def sync(self):
        from . import wave2d as w
        w.check(w.lib().wave2d_sync(self.sim.handle))
