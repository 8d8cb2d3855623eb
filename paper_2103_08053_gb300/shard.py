"""Workload partition across ranks (Sec. 5.1, the multi-GPU workload split).

Every rank holds the whole CSR and counts only the vertices u with
u % world == rank (``tc_params.shard_count`` / ``shard_index``: the counting
kernels skip the other vertices, orientation is replicated). The exchange is
one 64-bit sum of the per-rank counts; the step time of the job is the max of
the per-rank times. Both go through ``torch.distributed`` (NCCL on GPUs, gloo
on CPU), outside the counting path.
"""
from __future__ import annotations


def shard_params(rank: int, world: int) -> dict:
    """tc_params fields that restrict a context to rank's share of the vertices."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return {"shard_count": world, "shard_index": rank}


def owns(u: int, rank: int, world: int) -> bool:
    """The vertex-to-rank rule the kernels apply."""
    return u % world == rank


def combine(count: int, ms: float, device=None, group=None) -> tuple[int, float]:
    """(sum of the ranks' counts, max of the ranks' times); the identity when
    no process group is initialised or it has one rank."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return int(count), float(ms)
    if count < 0 or count >= 1 << 63:
        raise ValueError("a per-rank count must fit in int64 for the sum")
    dev = device if device is not None else torch.device("cpu")
    c = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return int(c.item()), float(t.item())
