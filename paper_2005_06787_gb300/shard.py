"""Slice-range sharding across processes (one GPU each).

Subtasks (slices) are independent and their values add (Supp. A.1
"Slicing"; Supp. A.4: subtasks need no communication). Each rank takes one
contiguous block of the slice range; the only exchange is the final sum of
the few (n_prefixes * 2^n_open) FP64 amplitudes, outside the contraction.
"""

from __future__ import annotations

from typing import Tuple


def slice_range(rank: int, world: int, total: int, begin: int = 0) -> Tuple[int, int]:
    """Half-open block of [begin, begin + total) owned by `rank` of `world`:
    sizes differ by at most one, lower ranks take the larger blocks."""
    if world <= 0 or not 0 <= rank < world or total < 0:
        raise ValueError("bad rank / world / total")
    q, r = divmod(total, world)
    lo = begin + rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def all_reduce_amplitudes(t, group=None):
    """Sum a float64 tensor of partial amplitudes over the process group
    (in place) and return it."""
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
