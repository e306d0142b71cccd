"""The loop contraction of one point split over ranks (one GPU per rank).

The loops of different transfer momenta l are independent (Eq. chis at each
l; the paper distributes the bosonic momenta over its MPI ranks, Sec. 3).
Here the unit of work is the loop row -- one per class of l under the
point-group elements that map l into the zone without a fold -- and rank r
computes the rows [r0, r1) of a contiguous partition.  Once per right-hand
side the row loops of all ranks are all-gathered (one collective of
2 * nrow * npair doubles, padded to equal chunks); the state stays
replicated, so the projections and the products then run on every rank in
full, and every rank holds the whole derivative.

``row_partition``, ``row_classes`` and ``gather_rows`` are host logic (no
GPU): they run, and are tested, with any torch.distributed backend.
``ShardedSolver`` drives the library's row-range entry points on the current
CUDA device.
"""
from __future__ import annotations

import numpy as np

# the point group C4v as integer matrices acting on l in units of 2 pi / nc,
# in the library's order of elements
C4V = ((1, 0, 0, 1), (0, -1, 1, 0), (-1, 0, 0, -1), (0, 1, -1, 0), (1, 0, 0, -1),
       (-1, 0, 0, 1), (0, 1, 1, 0), (0, -1, -1, 0))


def row_partition(nrow: int, world: int) -> list[tuple[int, int]]:
    """Contiguous row ranges [r0, r1) of the ranks (sizes differ by one at most)."""
    return [(nrow * r // world, nrow * (r + 1) // world) for r in range(world)]


def row_classes(ncx: int, ncy: int, point_group: bool = True) -> list[list[tuple[int, tuple]]]:
    """The loop rows of a coarse grid: for each row the (l, g) it serves, its
    representative first (g the identity), l = ix * ncy + iy, g a 2x2 integer
    matrix as a row-major 4-tuple.  g ranges over C4v (square grids with a
    point-group adapted basis) or over {e, -1}, and serves l' = g l only when
    g l lies in the zone without a fold (the order of rows and of the (l, g)
    of a row is the library's)."""
    group = C4V if (point_group and ncx == ncy) else (C4V[0], C4V[2])
    hx, hy = ncx // 2, ncy // 2
    served = np.zeros(ncx * ncy, dtype=bool)
    rows = []
    for jx in range(ncx):
        for jy in range(ncy):
            if served[jx * ncy + jy]:
                continue
            ux, uy = jx - hx, jy - hy
            images = []
            for g in group:
                vx, vy = g[0] * ux + g[1] * uy, g[2] * ux + g[3] * uy
                if not (-hx <= vx < ncx - hx and -hy <= vy < ncy - hy):
                    continue
                lg = (vx + hx) * ncy + (vy + hy)
                if served[lg]:
                    continue
                served[lg] = True
                images.append((lg, g))
            rows.append(images)
    return rows


def gather_rows(rows, parts, rank, dist, group=None):
    """All-gather of the row loops: rows is a [2][nrow][npair] tensor whose
    rows parts[rank] hold this rank's result; on return every rank's rows
    are filled in.  One all_gather of equal chunks [2][max rows][npair]."""
    import torch
    r0, r1 = parts[rank]
    width = max(b - a for a, b in parts)
    chunk = torch.zeros((2, width, rows.shape[2]), dtype=rows.dtype, device=rows.device)
    chunk[:, :r1 - r0] = rows[:, r0:r1]
    out = [torch.empty_like(chunk) for _ in parts]
    dist.all_gather(out, chunk, group=group)
    for (a, b), c in zip(parts, out):
        rows[:, a:b] = c[:, :b - a]
    return rows


class ShardedSolver:
    """A Solver whose loop contraction computes this rank's rows only; the
    right-hand side all-gathers the row loops (torch.distributed, NCCL on
    GPUs) and finishes the projections and products on every rank."""

    def __init__(self, solver, rank, world, dist=None, group=None):
        from . import _abi
        self.s, self.rank, self.world, self.dist, self.group = solver, rank, world, dist, group
        self.nrow, self.npair = _abi.tufrg_row_info(solver.ctx)
        self.parts = row_partition(self.nrow, world)
        r0, r1 = self.parts[rank]
        _abi.tufrg_shard_rows(solver.ctx, r0, r1)
        self._rows = None

    def rows(self, lam):
        """The row loops [2][nrow][npair] at scale lam, gathered over ranks."""
        import torch
        from . import _abi, _stream
        if self._rows is None:
            self._rows = torch.zeros((2, self.nrow, self.npair), dtype=torch.float64,
                                     device="cuda")
        _abi.tufrg_loop_rows(self.s.ctx, float(lam), self._rows.data_ptr(), _stream())
        if self.world > 1:
            gather_rows(self._rows, self.parts, self.rank, self.dist, self.group)
        return self._rows

    def rhs(self, lam, y, out=None):
        from . import _abi, _stream
        out = self.s.empty(3) if out is None else out
        rows = self.rows(lam)
        _abi.tufrg_rhs_from_rows(self.s.ctx, float(lam), rows.data_ptr(),
                                 self.s._check(y, 3), self.s._check(out, 3), _stream())
        return out
