"""One grid split into column strips (fv_set_partition / fv_part_* of fv.h).

Each strip is a handle on its owned columns plus a 2-column halo on each inner
side; after every step the strips exchange the largest signal rate (dt of the
next step, reading R-cfl) and the two columns next to each inner side.  The
owned cells then hold bit for bit what one handle on the whole grid computes.

Two ways to run it:

* ``StripSolver(case, prec, parts)``: all strips in this process on the current
  GPU; the rates are reduced by fv_part_set_rate over one device array and each
  halo buffer is written by one strip's pack and read by its neighbour's
  unpack (no copies);
* ``DistributedStrip(case, prec, group)``: this rank's strip of a grid split
  over the ranks of a torch.distributed process group (one GPU per rank): the
  rate is all-reduced (max) and the halo buffers are sent and received between
  neighbouring ranks.

The rank exchange (``exchange_dist``) works on any object with the strip
protocol (``step``, ``rate_into``, ``set_rate``, ``pack``, ``unpack``,
``halo_buffer``, ``has_w``, ``has_e``), so that its bookkeeping can run on CPU
ranks with stand-in strips.  Everything numerical happens in libfv.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

HALO = 2


def split_columns(nx: int, parts: int):
    """Owned column ranges [a, b) of ``parts`` strips of an nx-column grid,
    as equal as possible, each at least HALO columns wide."""
    if parts < 1 or nx < HALO * parts:
        raise ValueError(f"cannot split {nx} columns into {parts} strips of >= {HALO} columns")
    edges = [round(k * nx / parts) for k in range(parts + 1)]
    return [(edges[k], edges[k + 1]) for k in range(parts)]


def strip_extent(nx: int, a: int, b: int):
    """Columns [lo, hi) of the grid held by the strip owning [a, b) and its
    owned range within them."""
    lo = a - HALO if a > 0 else 0
    hi = b + HALO if b < nx else nx
    return lo, hi, a - lo, b - lo


def strip_case(case, a: int, b: int):
    """The case of the strip owning columns [a, b): its columns with halos,
    shifted origin, solid mask and state; the grid's W/E boundary kinds on the
    grid's own sides, a wall on inner sides (their halo columns are replaced
    after every step, so the kind does not matter)."""
    lo, hi, _, _ = strip_extent(case.nx, a, b)
    sides = list(case.sides)
    if lo > 0:
        sides[0] = 0
    if hi < case.nx:
        sides[1] = 0
    sub = replace(case, nx=hi - lo, x0=case.x0 + lo * case.dx, sides=tuple(sides),
                  name=f"{case.name}_cols{a}-{b}")
    sub.solid = np.ascontiguousarray(case.solid[:, lo:hi])
    sub.q = np.ascontiguousarray(case.q[:, :, lo:hi])
    return sub


class Strip:
    """One strip: a libfv handle with its owned range set, plus its halo and
    rate buffers (device tensors)."""

    def __init__(self, case, prec: int, a: int, b: int, stream=None):
        import torch
        from . import fv
        self.fv = fv
        self.a, self.b = a, b
        self.lo, self.hi, self.own_lo, self.own_hi = strip_extent(case.nx, a, b)
        self.case = strip_case(case, a, b)
        self.solver = fv.Solver(self.case, prec, stream)
        fv.fv_set_partition(self.solver.h, self.own_lo, self.own_hi)
        self.has_w = self.lo < a
        self.has_e = self.hi > b
        self.nbytes = fv.fv_part_halo_bytes(self.solver.h)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def halo_buffer(self):
        import torch
        return torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)

    def set_state(self, q_grid) -> None:
        self.solver.set_state(np.ascontiguousarray(q_grid[:, :, self.lo:self.hi]))

    def step(self, cfl: float) -> None:
        self.fv.fv_step(self.solver.h, 1, cfl)

    def rate_into(self, buf) -> None:
        self.fv.fv_part_rate(self.solver.h, buf)

    def set_rate(self, rates) -> None:
        self.fv.fv_part_set_rate(self.solver.h, rates)

    def pack(self, side: int, buf) -> None:
        self.fv.fv_part_pack(self.solver.h, side, buf)

    def unpack(self, side: int, buf) -> None:
        self.fv.fv_part_unpack(self.solver.h, side, buf)

    def owned_state(self):
        q = self.solver.get_state()
        return q[:, :, self.own_lo:self.own_hi]

    def close(self) -> None:
        self.solver.close()


def exchange_dist(strip, rank: int, world: int, dist, rate, send, recv, group=None) -> None:
    """Rate and halo exchange of this rank's strip with its neighbours:
    all-reduce(max) of the rate, then the halo buffers sent to and received
    from ranks rank-1 (W) and rank+1 (E) in one batch.  rate: one-element
    tensor; send/recv: {0: W buffer, 1: E buffer} for the sides that exist."""
    strip.rate_into(rate)
    dist.all_reduce(rate, op=dist.ReduceOp.MAX, group=group)
    strip.set_rate(rate)
    ops = []
    if strip.has_w:
        strip.pack(0, send[0])
        ops.append(dist.P2POp(dist.isend, send[0], rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, recv[0], rank - 1, group))
    if strip.has_e:
        strip.pack(1, send[1])
        ops.append(dist.P2POp(dist.isend, send[1], rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, recv[1], rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if strip.has_w:
        strip.unpack(0, recv[0])
    if strip.has_e:
        strip.unpack(1, recv[1])


class StripSolver:
    """A grid advanced as ``parts`` strips on the current GPU (same stream)."""

    def __init__(self, case, prec: int, parts: int, stream=None):
        import torch
        self.case = case
        self.ranges = split_columns(case.nx, parts)
        self.strips = [Strip(case, prec, a, b, stream) for a, b in self.ranges]
        dev = self.strips[0].device
        self._rates = torch.zeros(parts, dtype=torch.float64, device=dev)
        self.rates = [self._rates[k:k + 1] for k in range(parts)]
        self.bufs = [(self.strips[k].halo_buffer(), self.strips[k].halo_buffer())
                     for k in range(parts - 1)]

    def _exchange_rates(self) -> None:
        for s, r in zip(self.strips, self.rates):
            s.rate_into(r)
        for s in self.strips:
            s.set_rate(self._rates)

    def _exchange_halos(self) -> None:
        for k in range(len(self.strips) - 1):
            e_to_w, w_to_e = self.bufs[k]
            self.strips[k].pack(1, e_to_w)
            self.strips[k + 1].pack(0, w_to_e)
        for k in range(len(self.strips) - 1):
            e_to_w, w_to_e = self.bufs[k]
            self.strips[k + 1].unpack(0, e_to_w)
            self.strips[k].unpack(1, w_to_e)

    def set_state(self, q) -> None:
        for s in self.strips:
            s.set_state(q)
        self._exchange_rates()

    def step(self, n: int, cfl: float | None = None) -> None:
        cfl = self.case.cfl if cfl is None else cfl
        for _ in range(n):
            for s in self.strips:
                s.step(cfl)
            self._exchange_rates()
            self._exchange_halos()

    def get_state(self):
        return np.concatenate([s.owned_state() for s in self.strips], axis=2)

    def diag(self):
        """(t, steps, status) of the strips (equal t and steps on every strip)."""
        ds = [s.solver.diag() for s in self.strips]
        return ds[0].t, ds[0].steps, max(d.status for d in ds), [d.t for d in ds]

    def close(self) -> None:
        for s in self.strips:
            s.close()


class DistributedStrip:
    """This rank's strip of a grid split over the ranks of a process group
    (one strip per rank, in rank order from the W side)."""

    def __init__(self, case, prec: int, dist, group=None, stream=None):
        import torch
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.case = case
        a, b = split_columns(case.nx, self.world)[self.rank]
        self.strip = Strip(case, prec, a, b, stream)
        dev = self.strip.device
        self.rate = torch.zeros(1, dtype=torch.float64, device=dev)
        self.send = {k: self.strip.halo_buffer() for k in (0, 1)
                     if (self.strip.has_w if k == 0 else self.strip.has_e)}
        self.recv = {k: self.strip.halo_buffer() for k in self.send}

    def set_state(self, q_grid) -> None:
        self.strip.set_state(q_grid)
        self.strip.rate_into(self.rate)
        self.dist.all_reduce(self.rate, op=self.dist.ReduceOp.MAX, group=self.group)
        self.strip.set_rate(self.rate)

    def step(self, n: int, cfl: float | None = None) -> None:
        cfl = self.case.cfl if cfl is None else cfl
        for _ in range(n):
            self.strip.step(cfl)
            exchange_dist(self.strip, self.rank, self.world, self.dist, self.rate, self.send,
                          self.recv, self.group)

    def owned_state(self):
        return self.strip.owned_state()

    def close(self) -> None:
        self.strip.close()
