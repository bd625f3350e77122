"""A galaxy catalogue over several processes, one per GPU.

Galaxies are independent units of the method (Sec. 4 fits them in parallel
with no exchange), so each process takes a contiguous block of galaxies, runs
its own context on them, and the only collective is a host-side gather of the
results at the end.  The split itself is native (`sps_partition_galaxies`):
blocks balanced by the galaxies' observed bands plus a fixed part per galaxy.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from ._lib import check, load


def partition_galaxies(mask, n_parts: int, base_weight: int = 0) -> np.ndarray:
    """Block starts [n_parts + 1] (int64): block p is galaxies
    starts[p]:starts[p + 1].  A galaxy weighs base_weight (the fixed part of
    its cost, in units of one observed band's share) plus its observed bands;
    the heaviest block is made as light as possible.  mask: [n_gal] uint32
    band bitmasks (all zero: every galaxy weighs base_weight, and the counts
    are balanced when every weight is 0)."""
    lib = load()
    m = np.ascontiguousarray(np.asarray(mask), dtype=np.uint32)
    starts = np.zeros(int(n_parts) + 1 if n_parts >= 1 else 1, np.int64)
    check(lib.sps_partition_galaxies(C.c_void_p(m.ctypes.data), m.shape[0], int(base_weight),
                                     int(n_parts), C.c_void_p(starts.ctypes.data)),
          "sps_partition_galaxies")
    return starts


def block_of(mask, rank: int, world: int, base_weight: int = 0) -> tuple[int, int]:
    """[start, stop) of this process's galaxies."""
    s = partition_galaxies(mask, world, base_weight)
    return int(s[rank]), int(s[rank + 1])


def gather_blocks(local, dst: int = 0, group=None):
    """Host-side gather of per-galaxy results: every process passes its
    block's array (leading axis = its galaxies, any trailing shape); process
    dst receives the blocks concatenated in rank order, i.e. in catalogue
    order, the others None.  dst is a global rank (a member of group).  Uses
    torch.distributed's object gather, so with the NCCL backend each process
    must have selected its device first."""
    import torch.distributed as dist
    arr = np.asarray(local)
    world = dist.get_world_size(group)
    rank = dist.get_rank()
    parts = [None] * world if rank == dst else None
    dist.gather_object(arr, parts, dst=dst, group=group)
    if rank != dst:
        return None
    return np.concatenate(parts, axis=0)
