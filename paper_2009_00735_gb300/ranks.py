"""Host-side rank helpers for multi-process runs (one process per GPU).

ROIs are independent and the path has no exchange step, so ranks never
communicate on the data path: a multi-GPU run is a set of replicas (weak
scaling), or a contiguous split of one ROI list.  The only collectives are a
barrier and the max-over-ranks of a timing.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def roi_shard(nroi: int, rank: int, world: int):
    """Contiguous [lo, hi) share of nroi ROIs for `rank`; shares differ by at most one."""
    base, extra = divmod(nroi, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
