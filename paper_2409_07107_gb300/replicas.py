"""Replica parallelism across GPUs (host side only).

The environments of a batch are independent, so several GPUs simply run replicas: every rank
simulates its own seeded batch and nothing on the data path is exchanged.  The only collective is
the timing reduction of a benchmark: the job's time for a step is the slowest rank's, and the
job's throughput counts the envs of all ranks.
"""


def rank_seed(seed, rank):
    """Seed of rank `rank`'s batch (distinct per rank, reproducible)."""
    return int(seed) + 7919 * int(rank)


def slowest_ms(local_ms, group=None):
    """The maximum of `local_ms` over the ranks of the default (or given) process group; the value
    itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(local_ms)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(envs_per_rank, world, ms_per_step):
    """Env-steps per second of the whole job: all ranks' envs over the slowest rank's step time."""
    return float(envs_per_rank) * int(world) / (float(ms_per_step) * 1e-3)
