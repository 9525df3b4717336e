"""Host logic of the multi-GPU path, run as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1210_7683_gb300.sharding import (assemble, grid_rate, max_over_ranks, snp_shard, weak_scaling_rate,
                                            weak_shard)


@pytest.mark.parametrize("m,world", [(10, 3), (1000, 8), (7, 7), (0, 2), (5, 1)])
def test_shards_tile_the_range(m, world):
    ranges = [snp_shard(m, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == m
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import EigOracle
        from synth import covariates, genotypes, heritabilities, kinship, phenotypes
        # the bench's multi-rank layout: one problem of m_per_rank * world SNPs, each rank
        # generating and solving only its own shard (the oracle stands in for the GPU here)
        n, m_per_rank, t = 64, 19, 5
        m_total, i0, i1 = weak_shard(m_per_rank, rank, world)
        XR = genotypes(n, m_total, 12, i0=i0, i1=i1)
        b, se = EigOracle(kinship(n, 12), covariates(n, 3, 12)).solve(XR, phenotypes(n, t, 12), heritabilities(t, 12))
        # results are [traits][SNPs] like the library's LAST_SE output
        grid = assemble(np.stack([b[..., -1].T, se.T]), i0, i1, m_total)
        mx = max_over_ranks(10.0 + rank)
        results[rank] = (grid, mx, (i0, i1))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_grid():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        results = man.dict()
        mp.start_processes(_worker, args=(world, _free_port(), results), nprocs=world, start_method="spawn")
        got = dict(results)
    from oracle import EigOracle
    from synth import make_problem
    P = make_problem(64, 38, 5, seed=12)  # the whole problem the two shards belong to
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    assert sorted(got[r][2] for r in range(world)) == [(0, 19), (19, 38)]
    for rank in range(world):
        grid, mx, _ = got[rank]
        assert mx == 11.0
        assert grid.shape == (2, P.t, P.m)
        np.testing.assert_allclose(grid[0], b[..., -1].T, rtol=0, atol=1e-12)
        np.testing.assert_allclose(grid[1], se.T, rtol=0, atol=1e-12)
    assert weak_scaling_rate(100, 2, 500.0) == 400.0
    assert grid_rate(400, 500.0) == 800.0


def test_assemble_refuses_gaps_and_overlaps():
    blk = np.zeros((2, 3, 4))
    assert assemble(blk, 0, 4, 4).shape == (2, 3, 4)
    with pytest.raises(ValueError):
        assemble(blk, 1, 5, 5)       # a gap before the only shard
    with pytest.raises(ValueError):
        assemble(blk, 0, 4, 6)       # the shards end before the grid does
    with pytest.raises(ValueError):
        assemble(blk, 0, 3, 3)       # block width differs from its range
