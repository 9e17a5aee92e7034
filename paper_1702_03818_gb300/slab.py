"""One grid over several ranks: slabs of rows with halo rows exchanged between groups of stages.

A 2D grid that is periodic in y is split into one contiguous slab of rows per rank (heights
differing by at most one).  Each rank holds its slab extended by h halo rows on each side and
runs the stages on the extended slab as an ordinary periodic problem.  One stage moves
information one row, so after an exchange that makes the halo rows exact, m <= h stages leave
every interior row exact: the wrong values that the extended array's own wrap brings in start at
its two ends and move m rows inward at most.  Per group of m stages each rank sends its h bottom
interior rows to the rank below and its h top interior rows to the rank above (one message each
way per neighbour, into the receiver's own memory; no collective).  The conductivity's halo rows
are exchanged once.  ``slab_steps`` runs whole FRKC2 steps this way with ``frkc2_stages``
(Sec. 3, Eq. 13: a step is s stages W^{l+1} = W^l + T a_l f(W^l), so a step may stop after any
stage and resume there).

Host logic only: the stages run in the library's kernels; the messages go through
torch.distributed (NCCL with device tensors; gloo through host memory).
"""
from __future__ import annotations

import numpy as np


class Slab:
    """The rows of one rank: global rows [y0, y1) of a y-periodic grid of ny rows, held with
    ``halo`` rows on each side (extended row i is global row (y0 - halo + i) mod ny)."""

    def __init__(self, ny: int, world: int, rank: int, halo: int):
        if not (0 <= rank < world):
            raise ValueError("rank out of range")
        if halo < 1:
            raise ValueError("halo must be at least one row")
        self.ny, self.world, self.rank, self.h = int(ny), int(world), int(rank), int(halo)
        self.y0 = rank * ny // world
        self.y1 = (rank + 1) * ny // world
        self.n = self.y1 - self.y0
        if min((r + 1) * ny // world - r * ny // world for r in range(world)) < halo:
            raise ValueError("every slab must be at least `halo` rows high (the halo comes from one neighbour)")
        self.lower = (rank - 1) % world  # the rank holding the rows below this slab
        self.upper = (rank + 1) % world

    @property
    def rows_ext(self) -> int:
        return self.n + 2 * self.h

    def global_rows(self) -> np.ndarray:
        """Global row of every extended row."""
        return np.arange(self.y0 - self.h, self.y1 + self.h) % self.ny

    def interior(self) -> slice:
        return slice(self.h, self.h + self.n)

    def extend(self, a):
        """The extended slab of a global array (rows first), taken directly: for inputs that
        every rank holds, and for tests."""
        return a[self.global_rows()]


def exchange_halos(t, slab: Slab, group=None) -> None:
    """Fill the halo rows of ``t`` (a tensor whose first dimension is the extended slab's rows)
    from the neighbours: rows [0, h) with the lower neighbour's top h interior rows, rows
    [h + n, n + 2h) with the upper neighbour's bottom h interior rows.  Every rank sends its own
    interior rows the same way, so all ranks must call this together.  The four point-to-point
    operations are posted together (sends to the upper then the lower neighbour, receives from
    the lower then the upper one: with two ranks both messages of a pair go to the same peer
    and are matched in that order).  A backend that cannot move device tensors (gloo) gets host
    copies."""
    import torch
    import torch.distributed as dist

    h, n = slab.h, slab.n
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    if world != slab.world:
        raise ValueError("the slab was made for another number of ranks")
    if t.shape[0] != slab.rows_ext:
        raise ValueError("tensor rows do not match the extended slab")
    if world == 1:  # the grid's own periodic wrap
        t[:h] = t[n:n + h]
        t[h + n:] = t[h:2 * h]
        return
    host = t.is_cuda and dist.get_backend(group) != "nccl"
    src = t.cpu() if host else t
    up = src[n:n + h].contiguous()        # top interior rows -> the upper neighbour's bottom halo
    down = src[h:2 * h].contiguous()      # bottom interior rows -> the lower neighbour's top halo
    lo = torch.empty_like(up)
    hi = torch.empty_like(up)
    rank_of = (lambda r: dist.get_global_rank(group, r)) if group is not None else (lambda r: r)
    ops = [dist.P2POp(dist.isend, up, rank_of(slab.upper), group),
           dist.P2POp(dist.isend, down, rank_of(slab.lower), group),
           dist.P2POp(dist.irecv, lo, rank_of(slab.lower), group),
           dist.P2POp(dist.irecv, hi, rank_of(slab.upper), group)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    if host:
        t[:h].copy_(lo)
        t[h + n:].copy_(hi)
    else:
        t[:h] = lo
        t[h + n:] = hi


def slab_steps(plan, s: int, nsteps: int, w_ext, slab: Slab, stages, stages_per_exchange: int | None = None,
               group=None, exchange=exchange_halos):
    """``nsteps`` FRKC2 steps of s stages on this rank's extended slab ``w_ext`` (interleaved
    complex state, rows first).  Before each group of m <= h stages (m = h by default) the halo
    rows are exchanged; ``stages(l0, l1)`` then applies stages l0 .. l1-1 to the whole extended
    slab in place (``frkc2_stages`` on the device; a step's first group starts from the real
    part).  Returns the number of exchanges."""
    m = stages_per_exchange or slab.h
    if not (1 <= m <= slab.h):
        raise ValueError("stages per exchange must lie in 1..halo")
    count = 0
    for _ in range(nsteps):
        l0 = 0
        while l0 < s:
            l1 = min(s, l0 + m)
            exchange(w_ext, slab, group)
            count += 1
            stages(l0, l1)
            l0 = l1
    return count


def device_stages(F, plan, prob_ext, dt, w_ext, ws, stream=None):
    """The ``stages`` callable of ``slab_steps`` for the library: frkc2_stages on the extended
    slab's problem (a periodic nx x (n + 2h) grid)."""
    def run(l0, l1):
        F.frkc2_stages(plan, prob_ext, dt, l0, l1, w_ext, ws, stream=stream)
    return run
