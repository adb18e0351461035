"""Host-side multi-rank helpers (one process per GPU).

The codec path shards without any data exchange: every 4^d block, and so
every message of a plan, is coded independently (Sec. II-C), so N GPUs either
each run their own field (weak scaling) or split one plan's messages between
them (strong scaling).  torch.distributed is used only for the barrier
around the timed region and the max-over-ranks of the elapsed time -- never
on the data path.
"""
import os

import torch
import torch.distributed as dist


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend=None):
    ws, rank, local = env()
    if ws > 1 and not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x, device="cpu"):
    """Largest value of x over all ranks (the slowest rank sets the time)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device="cpu"):
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(n_items, rank, world):
    """Contiguous [lo, hi) share of n_items for `rank` (strong scaling):
    sizes differ by at most one, every item owned exactly once."""
    base, rem = divmod(n_items, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def weak_throughput(units_per_rank, seconds_max, world):
    """Whole-job throughput when every rank processes the same work."""
    return units_per_rank * world / seconds_max


def finalize():
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
