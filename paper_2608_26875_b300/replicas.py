"""Right-hand-side sharding across ranks (one process per GPU).

Incidences (right-hand sides) are independent: every rank holds the whole geometry, applies or
solves its own contiguous block of columns with no exchange during the mat-vecs, and the
results meet only once, in a final gather.  These helpers hold the host-side logic so that it
can be checked with gloo ranks on CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def rhs_shard(n: int, rank: int, world: int) -> range:
    """Contiguous block of column indices owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (step times are reported as the slowest rank's)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_columns(local: torch.Tensor, n: int, dim: int = -1) -> torch.Tensor:
    """Reassemble the full set of n columns from every rank's shard (along `dim`) on all ranks."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    world = dist.get_world_size()
    sizes = [len(rhs_shard(n, r, world)) for r in range(world)]
    dim = dim % local.dim()
    if local.shape[dim] != sizes[dist.get_rank()]:
        raise ValueError(f"rank {dist.get_rank()} holds {local.shape[dim]} columns, its shard of {n} has "
                         f"{sizes[dist.get_rank()]}")
    # all_gather wants equal shapes: pad every shard to the largest, then trim
    big = max(sizes)
    shape = list(local.shape)
    shape[dim] = big
    padded = torch.zeros(shape, dtype=local.dtype, device=local.device)
    padded.narrow(dim, 0, local.shape[dim]).copy_(local)
    parts = [torch.empty_like(padded) for _ in range(world)]
    if local.is_complex():
        dist.all_gather([torch.view_as_real(p) for p in parts], torch.view_as_real(padded))
    else:
        dist.all_gather(parts, padded)
    return torch.cat([p.narrow(dim, 0, s) for p, s in zip(parts, sizes)], dim=dim)
