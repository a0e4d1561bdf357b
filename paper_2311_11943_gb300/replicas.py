"""Host logic of multi-GPU runs: one process per GPU, each factorising its own independent
problems (replicas of one coded QR, or its own shard of a batch of instances).  There is no
data-path collective; the only exchange is the max over ranks of the measured times, so that
the whole-job throughput is (sum of every rank's flops) / (slowest rank's time).
"""
import os


def rank_env():
    """(world size, rank, local rank) from the torch.distributed launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(seed, rank):
    """Seed of rank `rank`'s inputs: the ranks factorise independent draws of one recipe."""
    return seed + 7919 * rank


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise max of a list of floats over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(flops_per_rank, world, ms_max):
    """Whole-job TFLOP/s: every rank did flops_per_rank in at most ms_max milliseconds."""
    return world * flops_per_rank / (ms_max * 1e-3) / 1e12
