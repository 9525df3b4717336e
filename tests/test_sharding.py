"""Host logic of the multi-GPU path, run as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1210_7683_gb300.sharding import max_over_ranks, snp_shard, weak_scaling_rate


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
        from synth import make_problem
        P = make_problem(64, 37, 5, seed=12)
        i0, i1 = snp_shard(P.m, rank, world)
        b, se = EigOracle(P.phi, P.XL).solve(P.XR[i0:i1], P.Y, P.h2)
        parts = [None] * world
        dist.all_gather_object(parts, (i0, i1, b, se))
        mx = max_over_ranks(10.0 + rank)
        results[rank] = (parts, mx)
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
    P = make_problem(64, 37, 5, seed=12)
    b, se = EigOracle(P.phi, P.XL).solve(P.XR, P.Y, P.h2)
    for rank in range(world):
        parts, mx = got[rank]
        assert mx == 11.0
        parts = sorted(parts)
        assert parts[0][0] == 0 and parts[-1][1] == P.m
        np.testing.assert_allclose(np.concatenate([p[2] for p in parts]), b, rtol=0, atol=1e-12)
        np.testing.assert_allclose(np.concatenate([p[3] for p in parts]), se, rtol=0, atol=1e-12)
    assert weak_scaling_rate(100, 2, 500.0) == 400.0
