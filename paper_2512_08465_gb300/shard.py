"""Host logic of the multi-GPU forms (Section III: scenarios are independent).

Sharded single network (what bench.py runs under torchrun): every rank holds a
replica of the network; the unordered pairs (and the single outages) are split
into contiguous equal blocks, one per rank; each rank
fills the entries of its block in its own severity tables (255 elsewhere = not
evaluated), and one element-wise minimum over ranks merges them (0 and 1 are
below 255, and no pair is evaluated by two ranks).  The Risk Index of the
merged tables is then the single-rank one, bit for bit, because its reduction
is exact and order-independent.  Works with any torch.distributed backend
(gloo on CPU tensors, NCCL on device tensors).  The step time of a run is the
maximum over ranks.
"""
from __future__ import annotations

import numpy as np

MISSING = 255


def pair_block(rank: int, world: int, total: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous block of `total` items, sizes differing by at most one."""
    if not (0 <= rank < world) or total < 0:
        raise ValueError("bad rank, world or total")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the step time of a replicas run)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def merge_severity_device(table, group=None):
    """In-place element-wise minimum over ranks of a uint8 severity tensor (any device;
    one all-reduce).  A no-op on one rank.  gloo reduces an int32 copy."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return table
    if dist.get_backend(group) == "gloo":
        t = table.to(torch.int32)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
        table.copy_(t.to(torch.uint8))
    else:
        dist.all_reduce(table, op=dist.ReduceOp.MIN, group=group)
    return table


def merge_severity(table: np.ndarray, group=None) -> np.ndarray:
    """Element-wise minimum over ranks of a uint8 severity table (255 = not evaluated)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(table, dtype=np.int32))
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return t.numpy().astype(np.uint8)
