"""Replicas across GPUs: the decoder's shots are independent, so N ranks
decode disjoint shot ranges with no collective on the data path; only the
final reductions (max of the timed seconds, sum of the failure counts) cross
ranks.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
import torch


def shot_offset(rank, n_batches, batch, b):
    """First sampler shot index of batch b of `rank` (ranks own disjoint,
    contiguous ranges of n_batches * batch shots)."""
    return (rank * n_batches + b) * batch


def _reduce(x, op, device):
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64 if isinstance(x, float) else torch.int64, device=device)
    dist.all_reduce(t, op=op)
    return t.item()


def max_over_ranks(x, device="cpu"):
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x, device="cpu"):
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM, device)
