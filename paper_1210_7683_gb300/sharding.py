"""Multi-GPU sharding of the GLS grid (host logic only).

The (SNP, trait) pairs are independent (Fig. 1), so the grid shards by SNP range
with no exchange on the data path: every rank holds its own genotype shard and
solves all traits for it.  The only collectives are for timing: a barrier and the
maximum of the per-rank times.
"""
from __future__ import annotations


def snp_shard(m: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous SNP range [i0, i1) of `rank`; the ranges tile [0, m), sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world or m < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(m, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of `value` over the ranks of the default (or given) process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def weak_scaling_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)
