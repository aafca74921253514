"""Image-parallel replicas: the funnel transform shards by image with no
exchange on the data path (every image is independent).  Used by bench.py
under torchrun; the host logic runs the same with the gloo backend on CPU.

* ``shard(rank, world, per_rank)``: the image indices a rank owns (weak scaling:
  every rank gets ``per_rank`` images of its own).
* ``barrier()`` / ``max_over_ranks(x)``: the timed region is bracketed by
  barriers and the slowest rank's time is the job's time.
"""
from __future__ import annotations

import os
from typing import Tuple


def env_world() -> Tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(rank: int, world: int, per_rank: int) -> range:
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank / world / per_rank")
    return range(rank * per_rank, (rank + 1) * per_rank)


def init(backend: str, device=None) -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        return
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    if device is not None and backend == "nccl":
        dist.init_process_group(backend, device_id=device)
    else:
        dist.init_process_group(backend)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def finish() -> None:
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
