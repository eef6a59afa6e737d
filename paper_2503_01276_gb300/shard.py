"""One hierarchy split over several ranks (one GPU per rank).

The macropoints of a level are independent (Algorithm 1, lines 4-6): each one needs only
the cell functions of its parents on earlier levels (Eq. phiXiI_all). So every level is cut
into contiguous point ranges, one per rank; a rank solves its range of a level
(mch_solve_level_range), then the ranks exchange that level's cell functions (the one
exchange step per level: an all-gather through host memory, no device-to-device multicast),
and every rank imports the other ranges (mch_set_cell_functions) before the next level. The
effective coefficients are gathered at the end. Points of one level cost the same
((n_level - 1)^d interior nodes times R functions), so equal point counts balance the work.

The backward pass is not split: mch_backward needs a handle that solved every point.

A backend does the per-rank work (``LibraryBackend`` wraps a ``Solver``); a communicator
provides ``allgather(obj) -> list over ranks`` (``TorchComm`` uses torch.distributed).
"""
from __future__ import annotations

import numpy as np


def partition(n_points: int, world: int):
    """Contiguous ranges [p0, p1) of a level's points, one per rank: equal sizes, the first
    n_points % world ranks one point more."""
    base, extra = divmod(int(n_points), int(world))
    out, p = [], 0
    for r in range(world):
        c = base + (1 if r < extra else 0)
        out.append((p, p + c))
        p += c
    return out


class LibraryBackend:
    """Per-rank work through the library handle of this rank's GPU."""

    def __init__(self, solver):
        self.s = solver

    def num_points(self, level):
        return self.s.num_points(level)

    def solve_range(self, level, p0, p1, kappa, labels):
        self.s.solve_level_range(level, p0, p1, kappa, labels)

    def cell_functions(self, level, p0, p1):
        return np.ascontiguousarray(self.s.cell_functions(level)[p0:p1])

    def set_cell_functions(self, level, p0, p1, phi):
        self.s.set_cell_functions(level, p0, p1, np.ascontiguousarray(phi))

    def effective_coeffs(self, level, p0, p1):
        return np.ascontiguousarray(self.s.effective_coeffs(level)[p0:p1])


class TorchComm:
    """All-gather of host objects over a torch.distributed process group (gloo or NCCL)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def allgather(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out


class ShardedHierarchy:
    """This rank's part of a hierarchy of ``n_levels`` levels split over ``world`` ranks.

    media(level, p0, p1) -> (kappa, labels) of points [p0, p1) of the level."""

    def __init__(self, backend, n_levels: int, world: int, rank: int, media):
        self.b = backend
        self.L = int(n_levels)
        self.world, self.rank = int(world), int(rank)
        self.media = media
        self.ranges = [partition(backend.num_points(l), world) for l in range(1, self.L + 1)]

    def own(self, level):
        return self.ranges[level - 1][self.rank]

    def solve_own(self, level):
        """Solves this rank's range of the level; returns (p0, p1, cell functions of the
        range) for the exchange (None on the last level, whose functions no child reads)."""
        p0, p1 = self.own(level)
        if p1 > p0:
            k, lb = self.media(level, p0, p1)
            self.b.solve_range(level, p0, p1, k, lb)
        else:
            self.b.solve_range(level, p0, p1, None, None)
        if level == self.L:
            return None
        phi = self.b.cell_functions(level, p0, p1) if p1 > p0 else None
        return (p0, p1, phi)

    def import_level(self, level, gathered):
        """Imports the other ranks' cell functions of the level (the exchange step)."""
        for r, item in enumerate(gathered):
            if r == self.rank or item is None:
                continue
            q0, q1, phi = item
            if q1 > q0:
                self.b.set_cell_functions(level, q0, q1, phi)

    def own_coeffs(self):
        out = []
        for level in range(1, self.L + 1):
            p0, p1 = self.own(level)
            out.append((p0, p1, self.b.effective_coeffs(level, p0, p1) if p1 > p0 else None))
        return out

    def run(self, comm):
        """Every level in order with its exchange step; returns the whole hierarchy's
        effective coefficients per level (gathered on every rank)."""
        for level in range(1, self.L + 1):
            item = self.solve_own(level)
            if level < self.L:
                self.import_level(level, comm.allgather(item))
        return assemble(comm.allgather(self.own_coeffs()), self.L)


def assemble(per_rank, n_levels):
    """Effective coefficients per level from every rank's (p0, p1, E) ranges."""
    out = []
    for lv in range(n_levels):
        parts = sorted((p0, p1, E) for rk in per_rank for (p0, p1, E) in [rk[lv]] if p1 > p0)
        out.append(np.concatenate([E for _, _, E in parts]) if parts else None)
    return out
