"""Slab-partitioned y = G x over torch.distributed (Sec. 2.7 and Algorithm 1).

Rank r holds the slab partition r of one mesh (cell layers bounds[r]..bounds[r+1]
along the last axis, see gp_partition_slabs / gp_partition_info).  Its local
vector is the global vector restricted to its lattice planes plus one cell of
halo above, so both exchanges of Algorithm 1 are one contiguous block between
neighbouring ranks:

  import_halo   x_local[n_owned:] on rank r  <-  x_local[:n_lower] of rank r + 1
                (ghost values of u, before the face loop);
  export_add    y_local[:n_lower] of rank r + 1  +=  y_local[n_owned:] of rank r
                (contributions to ghost entries, after it).

Point-to-point messages with the two neighbours only; no collective.  The
tensors may be CPU tensors (gloo) or CUDA tensors (NCCL).  After export_add,
y_local[:n_owned] equals the owned block of the global y; the halo entries of
y_local keep only this rank's own contributions.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import gp


def _neighbours(group):
    rank = dist.get_rank(group)
    return rank, dist.get_world_size(group)


def _global(group, r):
    return r if group is None else dist.get_global_rank(group, r)


def import_halo(x_local: torch.Tensor, info: dict, group=None) -> None:
    """Fill x_local[n_owned:] with the owned values of the partition above."""
    rank, ws = _neighbours(group)
    n_owned, n_local, n_lower = info["n_owned"], info["n_local"], info["n_lower"]
    reqs = []
    if rank + 1 < ws and n_local > n_owned:
        reqs.append(dist.irecv(x_local[n_owned:n_local], src=_global(group, rank + 1), group=group))
    if rank > 0 and n_lower > 0:
        reqs.append(dist.isend(x_local[:n_lower], dst=_global(group, rank - 1), group=group))
    for r in reqs:
        r.wait()


def export_add(y_local: torch.Tensor, info: dict, group=None) -> None:
    """Add the halo block of the partition below into y_local[:n_lower]."""
    rank, ws = _neighbours(group)
    n_owned, n_local, n_lower = info["n_owned"], info["n_local"], info["n_lower"]
    reqs, buf = [], None
    if rank > 0 and n_lower > 0:
        buf = torch.empty(n_lower, dtype=y_local.dtype, device=y_local.device)
        reqs.append(dist.irecv(buf, src=_global(group, rank - 1), group=group))
    if rank + 1 < ws and n_local > n_owned:
        reqs.append(dist.isend(y_local[n_owned:n_local], dst=_global(group, rank + 1), group=group))
    for r in reqs:
        r.wait()
    if buf is not None:
        y_local[:n_lower] += buf


class SlabOperator:
    """This rank's slab of y = G x for a workloads.Problem (one rank per partition)."""

    def __init__(self, pr, precision: int = gp.GP_FP64, device: int = 0, bounds=None, group=None):
        rank, ws = _neighbours(group)
        self.bounds = gp.partition_problem(pr, ws) if bounds is None else bounds
        if len(self.bounds) != ws + 1:
            raise ValueError("one partition per rank")
        self.group = group
        self.ctx = gp.setup_problem(pr, precision, device, part=(self.bounds[rank], self.bounds[rank + 1]))
        self.info = gp.gp_partition_info(self.ctx)

    def apply(self, x_local: torch.Tensor, y_local: torch.Tensor, stream=None) -> None:
        """x_local[:n_owned] in, y_local[:n_owned] out; x_local's halo is overwritten."""
        import_halo(x_local, self.info, self.group)
        gp.gp_apply(self.ctx, x_local, y_local, stream)
        export_add(y_local, self.info, self.group)
