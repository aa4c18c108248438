"""Host side of a multi-GPU run: independent replicas.

The light-field path has no exchange step between GPUs: a frame's planes are
built and composited on one device. A run on N GPUs is therefore N
independent replicas, one process per GPU, each rendering its own seeded copy
of a workload of the same size. The only collectives are a barrier around the
timed region and the maximum of the per-rank times; the whole-job rate is the
frames of all ranks divided by the slowest rank's time ("weak" scaling: the
work per GPU is fixed as N grows).

The helpers take the default process group as given: NCCL on GPUs, gloo in
the CPU tests.
"""
import os
from typing import Optional, Tuple


def env_rank() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank's copy of the workload: distinct scenes, same sizes."""
    if rank < 0:
        raise ValueError("rank must be non-negative")
    return base + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Maximum of value over all ranks (the value itself when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device: Optional[object] = None) -> None:
    """Process barrier, then (on a GPU) a device synchronise."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if device is not None and getattr(device, "type", None) == "cuda":
        import torch
        torch.cuda.synchronize(device)


def job_rate(max_ms_per_step: float, world: int, units_per_step: float = 1.0) -> float:
    """Whole-job rate in units per second: every rank processed units_per_step
    per step, and the job advances at the slowest rank's max_ms_per_step."""
    if not max_ms_per_step > 0:
        raise ValueError("time per step must be positive")
    if world < 1:
        raise ValueError("world size must be at least 1")
    return 1000.0 / max_ms_per_step * units_per_step * world
