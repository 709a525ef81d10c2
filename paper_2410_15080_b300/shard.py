"""Sharding the slices of one contraction over ranks.

Slices (value assignments of the sliced indices) are independent: rank r of
w contracts a contiguous range of them with ``qtpu_htn_contract_slices`` and
one sum over ranks of the (small, FP64) outputs gives the full result.  This
is the path's only exchange step.
"""
from __future__ import annotations


def slice_range(rank: int, world: int, n_slices: int):
    """(first, count) of rank's share: contiguous, sizes differ by at most 1."""
    if not (0 <= rank < world) or n_slices < 0:
        raise ValueError("bad rank / world / n_slices")
    base, extra = divmod(n_slices, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)
