"""Visibility sharding of the operator over processes, one GPU each: the distribution the paper
sketches for several compute nodes (Sec. 4.4, last paragraphs).  The rows of the measurement set
are split evenly over the ranks; each rank plans and runs the operator on its own rows:

  * degrid (R): the image is broadcast from one rank, then every rank degrids its rows -- the
    visibilities stay distributed, rank r holding rows row_block(nrows, world, r);
  * grid (R^dagger): every rank grids its rows into a full image, and one all-reduce (sum) of
    the images gives every rank R^dagger of the whole data set (R^dagger is a sum over
    visibilities, Eq. adjnfft / Rad1).

Each rank's plan sees only its rows (its own w range, planes and kernel choice); the operator is
the same, and each partial result meets the requested accuracy, so the sum does too.  The
collectives are torch.distributed calls on the default (or a given) process group: NCCL with GPU
tensors, gloo with CPU tensors.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple


def row_block(nrows: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [r0, r1) of rank `rank` when `nrows` rows are split as evenly as possible."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world / rank")
    q, r = divmod(int(nrows), int(world))
    r0 = rank * q + min(rank, r)
    return r0, r0 + q + (1 if rank < r else 0)


class ShardedOperator:
    """R and R^dagger over the rows of all ranks of a process group.

    make_plan(uvw_rows, freq, npix_x, npix_y, pixsize_x, pixsize_y, epsilon, precision,
    **plan_opts) builds the per-rank operator (default: the library's Plan on this rank's GPU);
    it must offer degrid(image) and grid(vis)."""

    def __init__(self, uvw, freq, npix_x, npix_y, pixsize_x, pixsize_y, epsilon,
                 precision="f32", group=None, make_plan: Optional[Callable] = None, **plan_opts):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.nrows = int(uvw.shape[0])
        self.rows = row_block(self.nrows, self.world, self.rank)
        if make_plan is None:
            from .wgrid import Plan as make_plan
        r0, r1 = self.rows
        self.plan = make_plan(uvw[r0:r1], freq, npix_x, npix_y, pixsize_x, pixsize_y, epsilon,
                              precision, **plan_opts)

    def degrid(self, dirty, src: int = 0):
        """Broadcast the image from rank `src` (in place on every rank's `dirty`, which must
        have the image's shape and dtype), then degrid this rank's rows: returns this rank's
        (r1 - r0, nchan) visibilities."""
        self.dist.broadcast(dirty, src=src, group=self.group)
        return self.plan.degrid(dirty)

    def grid(self, vis_rows):
        """Grid this rank's rows (vis_rows: (r1 - r0, nchan)) and sum the images of all ranks:
        every rank returns R^dagger of the whole data set."""
        img = self.plan.grid(vis_rows)
        self.dist.all_reduce(img, op=self.dist.ReduceOp.SUM, group=self.group)
        return img
