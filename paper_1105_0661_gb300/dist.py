"""Multi-process helpers for running independent observations on several GPUs of one node.

The station-to-beam path has no exchange step: subbands (and whole observations) are independent,
so N GPUs run N independent shards with no data-path collective.  torch.distributed is used only
for a barrier around the timed region and the max/sum of per-rank numbers.
"""

from __future__ import annotations

import os


def env_rank():
    """(rank, local_rank, world_size) from the torchrun environment (single process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def init(backend: str):
    """Initialise the default process group when WORLD_SIZE > 1 (env:// rendezvous)."""
    import torch.distributed as dist
    rank, _, world = env_rank()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def reduce_scalar(x: float, op: str = "max", device=None) -> float:
    """Max or sum of a per-rank float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return float(x)
    dev = device if (device is not None and dist.get_backend() == "nccl") else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def shard_range(n: int, rank: int, world: int):
    """Contiguous block [lo, hi) of n independent units (e.g. subbands) owned by `rank`."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def finalize():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
