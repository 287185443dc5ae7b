"""Multi-process launch helpers: markets are independent, so each rank runs its
own contiguous range of global market indices and no data-path collective
exists.  The only collectives are a barrier and a max-reduction of the timing.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment, else (0, 1, 0)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard(w: dict, rank: int, world: int) -> dict:
    """Weak scaling: every rank simulates the full ensemble size on its own
    market range [rank*M, (rank+1)*M) of the global index space."""
    out = dict(w)
    out["params"] = dict(w["params"])
    out["market_base"] = int(w.get("market_base", 0)) + rank * int(w["M"])
    return out


def init(backend: str):
    import torch.distributed as dist
    rank, world, _ = rank_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def finalize():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
