"""Instance-level data parallelism across GPUs (one process per GPU).

Detection problems are independent (one per subcarrier and time slot), so every rank
detects its own shard and nothing is exchanged on the data path.  Only scalars are
combined after the timed region: the maximum step time over ranks and sums of error
counters.  These helpers work with the NCCL backend (CUDA tensors) and with gloo (CPU).
"""
import torch
import torch.distributed as dist


def shard_range(n_total, rank, world):
    """Contiguous [start, stop) of the instances owned by `rank`."""
    base, rem = divmod(n_total, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)


def _device():
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def _reduce(x, op, world, dtype):
    if world <= 1 or not dist.is_initialized():
        return x
    t = torch.tensor([x], dtype=dtype, device=_device())
    dist.all_reduce(t, op=op)
    return t.item()


def max_over_ranks(x, world):
    return _reduce(float(x), dist.ReduceOp.MAX, world, torch.float64)


def sum_over_ranks(x, world):
    return int(_reduce(int(x), dist.ReduceOp.SUM, world, torch.int64))
