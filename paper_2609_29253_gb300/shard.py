"""Splitting the operator over ranks (one process per GPU).

The forward operator A decomposes over transducer positions: row k of s = A x
depends only on position k (Alg. 1 assembles f_k per transducer), so ranks
that own disjoint position sets produce disjoint rows of s with no exchange.
The adjoint A^T s = sum_k A_k^T s_k (Alg. 5) is a sum over positions: ranks
that own disjoint position sets each produce a partial z, and one all-reduce
(sum) of the N-vector gives the whole adjoint.  Independent problems or
position batches need no exchange at all (weak scaling).

Nothing here computes the operator: it partitions index sets and sums the
ranks' partial results with torch.distributed.
"""
from __future__ import annotations

import math

import numpy as np


def shard_range(K: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous, balanced range [lo, hi) of K positions owned by rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} not in a world of {world}")
    base, extra = divmod(int(K), world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_workload(w, rank: int, world: int):
    """The workload restricted to this rank's positions (and its range)."""
    lo, hi = shard_range(w.K, rank, world)
    return w.with_tx(w.tx[lo:hi]), (lo, hi)


def angle_batches(n_angles: int, batch: int, rank: int, world: int, steps: int) -> list[np.ndarray]:
    """Rotation angles of each step for one rank: the angles are cut into
    batches of `batch`; rank r takes batches r, r + world, r + 2 world, ...
    (wrapping), so ranks never share a batch within one pass."""
    nb = max(1, n_angles // batch)
    out = []
    for i in range(steps):
        b = (rank + i * world) % nb
        out.append(np.arange(b * batch, (b + 1) * batch) * 2 * math.pi / n_angles)
    return out


def allreduce_adjoint(z_partial, group=None):
    """Sum the ranks' partial adjoints in place (one all-reduce of N values)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(z_partial, op=dist.ReduceOp.SUM, group=group)
    return z_partial
