"""Multi-GPU split of the batched factorization: one process per GPU, each
factoring the share of the matrices that abft_batched_partition assigns it
(longest processing time first on n^3/3), with the per-matrix statuses
gathered on the host afterwards.  Nothing is exchanged on the data path."""
import ctypes

import numpy as np

from . import abft


def partition(sizes, G):
    """(owner, load): the GPU of each matrix (int32) and each GPU's work."""
    n = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
    owner = np.zeros(len(n), dtype=np.int32)
    load = np.zeros(G, dtype=np.float64)
    L = abft.lib()
    rc = L.abft_batched_partition(len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), G,
                                  owner.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  load.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise abft.AbftError(rc, abft.strerror(rc))
    return owner, load


def shard_ids(owner, rank):
    """Global indices of the matrices of one GPU, in increasing order."""
    return np.flatnonzero(np.asarray(owner) == rank)


def gather_statuses(ids, status, count, group=None):
    """Gather every rank's (ids, status rows) to rank 0 over the host process
    group and return the full status table (count x fields, row i = matrix i)
    on rank 0, None on the other ranks.  Single process: the rows reordered."""
    import torch.distributed as dist
    ids = np.asarray(ids, dtype=np.int64)
    status = np.asarray(status)
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        parts = [(ids, status)]
    else:
        parts = [None] * dist.get_world_size(group) if dist.get_rank(group) == 0 else None
        dist.gather_object((ids, status), parts, dst=0, group=group)
        if dist.get_rank(group) != 0:
            return None
    full = np.full((count, status.shape[1] if status.ndim == 2 else 1), -1, dtype=status.dtype)
    seen = np.zeros(count, dtype=np.int64)
    for i, st in parts:
        full[i] = st
        seen[i] += 1
    if not np.all(seen == 1):
        raise RuntimeError("every matrix must be reported by exactly one rank")
    return full
