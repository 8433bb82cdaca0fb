"""One process per GPU, each an independent replica of the workload.

The vertices of different fields (or replicas) share nothing, so the path
shards without any data exchange: every rank computes its own fields and the
job's throughput is (units of all ranks) / (slowest rank's timed region).
The only collectives are host-side: a barrier around the timed region and
the max / sum reductions below (gloo on CPU, NCCL on GPUs).
"""
import os

import torch
import torch.distributed as dist


def rank_env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, device=None):
    """Join the process group when launched with more than one rank."""
    rank, world, _ = rank_env()
    if world > 1 and not dist.is_initialized():
        if device is not None:
            dist.init_process_group(backend, device_id=device)
        else:
            dist.init_process_group(backend)
    return rank, world


def barrier():
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(local_ms, local_units, device="cpu"):
    """Whole-job throughput of weakly scaled replicas: the sum of the units
    every rank processed divided by the slowest rank's time.
    Returns (max_ms, total_units, units_per_second)."""
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    max_ms, units = float(t.item()), float(u.item())
    return max_ms, units, units / (max_ms / 1e3)
