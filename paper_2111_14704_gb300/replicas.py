"""Host logic of the replica runs (one periodic box per GPU, no data-path
collective): per-rank seeds, the max-over-ranks timing reduction and the
whole-job throughput.  The only collective is the timing reduction, on
whatever process group is initialised (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def replica_seed(base: int, rank: int) -> int:
    """Each rank's box draws its packets and modes from its own seed."""
    return base + rank


def reduce_max(values, world: int, device="cpu"):
    """Element-wise maximum over ranks of a list of floats (identity for one rank)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(world: int, units_per_rank: int, steps: int, ms_max: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling)."""
    return world * units_per_rank * steps / (ms_max * 1e-3)
