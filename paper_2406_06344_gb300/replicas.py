"""Replica-parallel runs: one process per GPU, each running the whole path on its own inputs.

Nothing in the method needs an exchange between GPUs when every GPU builds its own TT and its
own factors, so a multi-GPU run is N independent replicas (weak scaling). The only cross-rank
traffic is this module's bookkeeping: per-rank input seeds, the total of the work units done,
the maximum of the device times, and contiguous ranges for splitting a batch of instances.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

SEED_STRIDE = 1000   # rank r draws its inputs from seed + SEED_STRIDE * r


@dataclass(frozen=True)
class RankInfo:
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    """Rank, world size and local rank from the torchrun environment (defaults: one process)."""
    env = os.environ if env is None else env
    return RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def replica_seed(seed: int, rank: int) -> int:
    """Seed of a generator on the given rank: rank 0 keeps the single-GPU seed."""
    return seed + SEED_STRIDE * rank


def shard(total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [lo, hi) share of `total` units for `rank`; shares differ by at most one."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def aggregate(units: float, ms: list, group=None):
    """(units summed over ranks, each entry of `ms` maximised over ranks).

    With one process (or torch.distributed not initialised) the inputs come back unchanged.
    The reduction runs on the process group's own device kind: CPU tensors for gloo, the
    current CUDA device for nccl.
    """
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return float(units), [float(m) for m in ms]
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    t = torch.tensor([float(m) for m in ms], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(u.item()), t.tolist()
