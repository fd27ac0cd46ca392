"""Multi-rank host logic on CPU: realization sharding and the fixed-order FP64 moment merge,
exercised with world_size 2 over gloo (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2604_07248_gb300.sharding import merge_moments, shard


def test_shard_partitions_every_unit_once():
    for total in (0, 1, 7, 16, 1000):
        for world in (1, 2, 3, 8):
            got = [list(shard(total, r, world)) for r in range(world)]
            flat = [x for g in got for x in g]
            assert flat == list(range(total))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard(5, 2, 2)


def _welford_block(x):
    return len(x), x.mean(axis=0), ((x - x.mean(axis=0)) ** 2).sum(axis=0)


def test_merge_matches_single_pass_statistics():
    rng = np.random.default_rng(0)
    x = rng.gamma(2.0, 3.0, size=(37, 5, 5)) + 1e4
    parts = [_welford_block(x[r]) for r in (shard(37, k, 4) for k in range(4))]
    n, mean, m2 = merge_moments(parts)
    assert n == 37
    assert np.max(np.abs(mean - x.mean(axis=0))) < 1e-10
    assert np.max(np.abs(m2 / n - x.var(axis=0))) < 1e-8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    from paper_2604_07248_gb300.sharding import gather_merge, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(1)
    data = rng.normal(5.0, 2.0, size=(21, 4, 4))  # every rank sees the same global data set
    mine = data[list(shard(21, rank, world))]
    res = gather_merge(len(mine), mine.mean(axis=0), ((mine - mine.mean(axis=0)) ** 2).sum(axis=0))
    if rank == 0:
        q.put((res[0], res[1].tolist(), res[2].tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_gather_merge_over_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    n, mean, m2 = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    data = np.random.default_rng(1).normal(5.0, 2.0, size=(21, 4, 4))
    assert n == 21
    assert np.max(np.abs(np.array(mean) - data.mean(axis=0))) < 1e-12
    assert np.max(np.abs(np.array(m2) / n - data.var(axis=0))) < 1e-12
