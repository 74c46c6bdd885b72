"""Independent replicas on several GPUs of one node (one process per GPU).

The lattice update itself never exchanges data between GPUs here: each rank
advances its own lattice (weak scaling).  The ranks only meet to line up the
timed region (barrier) and to take the slowest rank's time.  Launched by
torchrun, which sets RANK, WORLD_SIZE and LOCAL_RANK.
"""

from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world, backend="nccl", device=None):
    if world <= 1:
        return
    import torch.distributed as dist
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=device)
    else:
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cpu"):
    """Maximum of a per-rank float over all ranks (the job's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max


def finish(world):
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
