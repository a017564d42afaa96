"""Replica plumbing of the benchmark on several GPUs of one node.

The search does not exchange data between GPUs: with N processes (one per
GPU) each runs its own replica of the workload (the single-system workloads)
or its round-robin share of independent systems / requests (the batched and
served workloads).  The only collectives are the barrier around the timed
region and the max-over-ranks of the elapsed time, so the whole-job rate is
(units all ranks processed) / (slowest rank's time).
"""
import os


def rank_env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, world):
    """Join the process group when there is more than one rank."""
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cpu"):
    """Largest value of x over all ranks (x itself with one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device="cpu"):
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(items, world, rank):
    """This rank's round-robin share of independent work items."""
    return list(items)[rank::world]


def whole_job_rate(units_this_rank, seconds_this_rank, world, device="cpu"):
    """Units processed by all ranks divided by the slowest rank's time."""
    return sum_over_ranks(units_this_rank, world, device) / max_over_ranks(seconds_this_rank, world, device)


def finish(world):
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
