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


# ------------------------------------------------------------------------------------------------
# the same merge on real accumulators: a small version of the Monte Carlo workload (plane wave
# through screens with 3-level subharmonics), each rank running the oracle's Welford over its shard
# ------------------------------------------------------------------------------------------------
MC = dict(lam=1.55e-6, N=64, dx=4e-3, dz=[200.0] * 3, cn2=1e-14, seed=0x2604072482, R=16)


def _mc_intensity(r):
    import oracle as O

    md = O.medium(MC["lam"], MC["N"], MC["dx"], l0=5e-3, L0=10.0)
    phis = np.stack([O.make_screen(md, MC["cn2"], dz, 3, MC["seed"], s, r) for s, dz in enumerate(MC["dz"])])
    U = O.propagate(md, MC["dz"], phis, np.ones((MC["N"], MC["N"]), complex))
    return np.abs(U) ** 2


def _mc_chunk(reals):
    import oracle as O

    w = O.Welford((MC["N"], MC["N"]))
    for r in reals:
        w.update(_mc_intensity(r))
    return w


def _rank_main_mc(rank, world, port, q):
    import torch.distributed as dist

    from paper_2604_07248_gb300.sharding import gather_merge, shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _mc_chunk(shard(MC["R"], rank, world))
    res = gather_merge(w.n, w.mean, w.M2)
    if rank == 0:
        q.put((res[0], res[1].tobytes(), res[2].tobytes()))
    dist.barrier()
    dist.destroy_process_group()


def test_monte_carlo_moments_sharded_over_two_gloo_ranks():
    # Sec. 3.3 / S25 moments, sharded by realization (every Philox counter depends only on the global
    # realization index): the merged accumulators equal, bit for bit, one process merging the same
    # per-shard oracle accumulators in rank order, and agree with the oracle's own single-pass
    # Welford and its own pairwise merge to rounding.
    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main_mc, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    n, mean_b, m2_b = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    N = MC["N"]
    mean = np.frombuffer(mean_b, np.float64).reshape(N, N)
    m2 = np.frombuffer(m2_b, np.float64).reshape(N, N)
    parts = [_mc_chunk(shard(MC["R"], k, 2)) for k in range(2)]
    n1, mean1, m21 = merge_moments([(w.n, w.mean, w.M2) for w in parts])
    assert n == n1 == MC["R"]
    assert np.array_equal(mean, mean1) and np.array_equal(m2, m21)  # bit for bit
    si = (m2 / n) / mean ** 2
    assert np.array_equal(si, (m21 / n1) / mean1 ** 2)
    single = _mc_chunk(range(MC["R"]))  # one sequential Welford pass
    oracle_merge = parts[0]
    oracle_merge.merge(parts[1])
    for ref in (single, oracle_merge):
        assert np.max(np.abs(mean - ref.mean) / np.abs(ref.mean)) < 1e-12
        assert np.max(np.abs(si - ref.si_map()) / ref.si_map().max()) < 1e-10
    assert 0.0 < si.mean() < 1.0  # weak scintillation of a unit plane wave
