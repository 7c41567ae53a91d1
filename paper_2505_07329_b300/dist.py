"""Token sharding across ranks (one process per GPU).

Tokens are independent ciphertexts, so the hot path shards by token with the
public weights replicated on every rank and no collective on the data path
(each rank's outputs go back to their own clients).  The only collectives
are for timing: a barrier around the timed region and the maximum of the
ranks' elapsed times.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(total: int, rank: int, world_size: int) -> tuple[int, int]:
    """Contiguous token range [t0, t1) of `rank`: sizes differ by at most one,
    every token belongs to exactly one rank, and rank order is token order."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank/world size")
    base, extra = divmod(total, world_size)
    t0 = rank * base + min(rank, extra)
    return t0, t0 + base + (1 if rank < extra else 0)


def weak_scaling_range(tokens_per_rank: int, rank: int) -> tuple[int, int]:
    """Weak scaling: every rank takes the same number of tokens of a global
    batch of tokens_per_rank * world tokens."""
    return rank * tokens_per_rank, (rank + 1) * tokens_per_rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (no-op
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
