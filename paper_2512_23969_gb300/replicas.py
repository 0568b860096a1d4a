"""Replica bookkeeping for runs over several GPUs of one node.

Signatures are independent, so the multi-GPU form of the signer is replicas:
each rank signs its own batch on its own GPU and nothing is exchanged on the
data path.  Only the timing is combined: the job's step time is the slowest
rank's, and the job's rate counts every rank's signatures.  The reduction is
a host-side gloo all-reduce of one number per rank.
"""
import torch


def init_from_env():
    """(world_size, rank, local_rank) from the torchrun environment; joins a
    gloo process group when world_size > 1."""
    import os
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group("gloo")
    return ws, rank, local


def max_over_ranks(value):
    """The maximum of a float over all ranks (the value itself when alone)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(world_size, per_rank_count, steps, max_total_ms):
    """Whole-job signatures/s: every rank signed per_rank_count per step."""
    return world_size * per_rank_count * steps / (max_total_ms / 1e3)


def barrier():
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()
