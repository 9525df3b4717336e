"""Multi-GPU sharding of the GLS grid (host logic only).

The (SNP, trait) pairs are independent (Fig. 1), so the grid shards by SNP range
with no exchange on the data path: every rank holds its own contiguous shard of
one problem's genotypes, replicates the small per-trait inputs (Phi, X_L, Y, h^2)
and solves all traits for its shard through the same C calls as one GPU
(gwas_load_snps of the shard, then gwas_solve).  The only collectives are for
timing (a barrier and the maximum of the per-rank times) and for gathering
sampled results to check them.
"""
from __future__ import annotations

import numpy as np


def snp_shard(m: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous SNP range [i0, i1) of `rank`; the ranges tile [0, m), sizes differ by <= 1."""
    if world < 1 or not 0 <= rank < world or m < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(m, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def weak_shard(m_per_rank: int, rank: int, world: int) -> tuple[int, int, int]:
    """Weak scaling over one problem: the problem has m_per_rank * world SNPs and `rank` holds
    the shard snp_shard of it.  Returns (m_total, i0, i1)."""
    m_total = m_per_rank * world
    i0, i1 = snp_shard(m_total, rank, world)
    return m_total, i0, i1


def gather_blocks(local: np.ndarray, i0: int, group=None) -> list[tuple[int, int, np.ndarray]]:
    """Every rank's block of results for SNPs [i0, i0 + width) (the last axis of `local`), as
    (i0, i1, block) sorted by i0, on every rank of the default (or given) process group."""
    import torch.distributed as dist
    item = (int(i0), int(i0) + local.shape[-1], np.ascontiguousarray(local))
    if not dist.is_available() or not dist.is_initialized():
        parts = [item]
    else:
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, item, group=group)
    return sorted(parts, key=lambda p: p[0])


def assemble(local: np.ndarray, i0: int, i1: int, m_total: int, group=None) -> np.ndarray:
    """The full grid from every rank's block of SNPs [i0, i1) (the last axis of `local`),
    gathered on every rank of the default (or given) process group.  Raises when the
    gathered ranges do not tile [0, m_total) exactly."""
    if local.shape[-1] != i1 - i0:
        raise ValueError("block width differs from its SNP range")
    parts = gather_blocks(local, i0, group)
    end = 0
    for a, b, blk in parts:
        if a != end or blk.shape[-1] != b - a:
            raise ValueError(f"shards do not tile the SNP range at {a} (expected {end})")
        end = b
    if end != m_total:
        raise ValueError(f"shards end at {end}, the grid has {m_total} SNPs")
    return np.concatenate([p[2] for p in parts], axis=-1)


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


def grid_rate(units_total: int, max_ms: float) -> float:
    """Whole-job throughput of one grid split over the ranks: its units over the slowest rank's time."""
    return units_total / (max_ms / 1e3)
