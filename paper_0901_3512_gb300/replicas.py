"""Replica parallelism across ranks, one process per GPU.

The method's independent problems need no exchange step, so every rank solves
its own copy of the workload.  The job's time for a step is the slowest rank's,
the maximum over ranks.  The whole job's seconds per solved problem is that time
divided by the number of replicas.  Only torch.distributed's barrier and a MAX
all-reduce of one number per measurement are used (NCCL on GPUs, gloo in the
CPU tests); no data moves between ranks.
"""
import os

import torch
import torch.distributed as dist


def world_rank_local():
    """(WORLD_SIZE, RANK, LOCAL_RANK) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def init(backend: str, device=None):
    """Join the process group when launched with more than one rank."""
    world, rank, local = world_rank_local()
    if world > 1 and not dist.is_initialized():
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=device)
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier():
    if _active():
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest x over all ranks (x itself on a single rank)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if _active():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_solve(step_seconds_max: float, world: int) -> float:
    """Whole-job seconds per solved problem: `world` replicas finish in the slowest
    rank's step time."""
    return step_seconds_max / max(int(world), 1)


def finish():
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
